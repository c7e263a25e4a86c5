/* Explicit-loop FP64 pieces of the NLPR oracle (test infrastructure only).
 *
 * TEST INFRASTRUCTURE ONLY: called from oracle/cloops.py by the tests, the
 * smoke check and the CPU-baseline leg of the benchmark; never by the product.
 *
 * Plain C loops over (tau, k, pixel, band), written from the definitions:
 *   oracle_weights  : omega_{i tau} = exp(-||P_{i tau}(G)||_2^2 / h^2)   (Sec. II-B, eq. wts)
 *   oracle_latent   : Q = S(D_{tau k}X - Sigma, lambda2 omega / rho)      (eq. Qj_main)
 *                     Sigma <- Sigma - (D_{tau k}X - Q)                   (eq. dualvar3_main)
 *   oracle_dt_sum   : sum_{tau,k} D_{tau k}^T (Q + Sigma)                 (right side of
 *                                                                          eq. x_linear_system_main)
 * with D_{tau k}X(i,c) = X_c(i-k) - X_c(i-tau-k) (eq. differencemat) on the periodic
 * domain.  Images are (H, W, L) row-major; Q and Sigma are (|W|, |P|, H, W, L);
 * omega is (|W|, H, W).  W = [-S,S]^2 without (0,0) and P = [-K,K]^2, both row-major.
 */
#include <math.h>
#include <stddef.h>

static inline int wrap(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

static int n_search(int S) { return (2 * S + 1) * (2 * S + 1) - 1; }

static void search_offset(int S, int t, int* t1, int* t2) {
    int side = 2 * S + 1;
    int idx = t >= (side * side) / 2 ? t + 1 : t;   /* skip the centre (0,0) */
    *t1 = idx / side - S;
    *t2 = idx % side - S;
}

void oracle_weights(const double* G, int H, int W, int L, int K, int S, double h, double* omega) {
    int nW = n_search(S);
    for (int t = 0; t < nW; ++t) {
        int t1, t2;
        search_offset(S, t, &t1, &t2);
        #pragma omp parallel for schedule(static)
        for (int i1 = 0; i1 < H; ++i1) {
            for (int i2 = 0; i2 < W; ++i2) {
                double acc = 0.0;
                for (int k1 = -K; k1 <= K; ++k1) {
                    for (int k2 = -K; k2 <= K; ++k2) {
                        const double* a = G + ((size_t)wrap(i1 - k1, H) * W + wrap(i2 - k2, W)) * L;
                        const double* b = G + ((size_t)wrap(i1 - t1 - k1, H) * W + wrap(i2 - t2 - k2, W)) * L;
                        for (int c = 0; c < L; ++c) {
                            double diff = a[c] - b[c];
                            acc += diff * diff;
                        }
                    }
                }
                omega[((size_t)t * H + i1) * W + i2] = exp(-acc / (h * h));
            }
        }
    }
}

void oracle_latent(const double* X, const double* omega, double* Q, double* Sig,
                   int H, int W, int L, int K, int S, double lam2, double rho) {
    int nW = n_search(S), side = 2 * K + 1, nP = side * side;
    size_t plane = (size_t)H * W * L;
    for (int t = 0; t < nW; ++t) {
        int t1, t2;
        search_offset(S, t, &t1, &t2);
        for (int kk = 0; kk < nP; ++kk) {
            int k1 = kk / side - K, k2 = kk % side - K;
            double* q = Q + ((size_t)t * nP + kk) * plane;
            double* s = Sig + ((size_t)t * nP + kk) * plane;
            #pragma omp parallel for schedule(static)
            for (int i1 = 0; i1 < H; ++i1) {
                for (int i2 = 0; i2 < W; ++i2) {
                    double mu = lam2 * omega[((size_t)t * H + i1) * W + i2] / rho;
                    const double* xa = X + ((size_t)wrap(i1 - k1, H) * W + wrap(i2 - k2, W)) * L;
                    const double* xb = X + ((size_t)wrap(i1 - t1 - k1, H) * W + wrap(i2 - t2 - k2, W)) * L;
                    size_t base = ((size_t)i1 * W + i2) * L;
                    for (int c = 0; c < L; ++c) {
                        double dx = xa[c] - xb[c];
                        double v = dx - s[base + c];
                        double mag = fabs(v) - mu;
                        double qn = mag > 0.0 ? (v > 0.0 ? mag : -mag) : 0.0;
                        q[base + c] = qn;
                        s[base + c] = s[base + c] - (dx - qn);
                    }
                }
            }
        }
    }
}

void oracle_dt_sum(const double* Q, const double* Sig, int H, int W, int L, int K, int S,
                   double* out) {
    int nW = n_search(S), side = 2 * K + 1, nP = side * side;
    size_t plane = (size_t)H * W * L;
    #pragma omp parallel for schedule(static)
    for (int i1 = 0; i1 < H; ++i1) {
        for (int i2 = 0; i2 < W; ++i2) {
            double* o = out + ((size_t)i1 * W + i2) * L;
            for (int c = 0; c < L; ++c) o[c] = 0.0;
            for (int t = 0; t < nW; ++t) {
                int t1, t2;
                search_offset(S, t, &t1, &t2);
                for (int kk = 0; kk < nP; ++kk) {
                    int k1 = kk / side - K, k2 = kk % side - K;
                    size_t off = ((size_t)t * nP + kk) * plane;
                    size_t pa = ((size_t)wrap(i1 + k1, H) * W + wrap(i2 + k2, W)) * L;
                    size_t pb = ((size_t)wrap(i1 + k1 + t1, H) * W + wrap(i2 + k2 + t2, W)) * L;
                    for (int c = 0; c < L; ++c)
                        o[c] += (Q[off + pa + c] + Sig[off + pa + c]) - (Q[off + pb + c] + Sig[off + pb + c]);
                }
            }
        }
    }
}
