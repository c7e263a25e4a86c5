// Reverse pass of one unrolled ADMM iteration (differentiation of the updates of Sec. IV).
//
// Forward iteration t, in the variables the solver keeps (state in: Lambda1, U1 = P1 + Lambda1,
// Lambda2, U2 = P2 + Lambda2, the latent state Sigma and the adjoint sum R of the previous pass):
//   C = B^T U1 + U2 + R,  X = A^{-1} C  (eq. inv),  BX = B X,
//   pixel (eqs. Qm_update, Qh_update, dualvar1_main, dualvar2_main):
//     w2 = X - Lambda2, a2 = w2 + D9b, P2 = a2 F, Lambda2' = P2 - w2, U2' = 2 P2 - w2,
//     w1 = BX - Lambda1, P1 = (rho w1 + D9a) M1 where sampled, else w1,
//     Lambda1' = P1 - w1, U1' = 2 P1 - w1;
//   latent (eqs. Qj_main, dualvar3_main), per offset tau and patch offset k:
//     v = D X - Sigma, Sigma' = -clamp(v, -mu, mu), G = v + 2 Sigma', R' = sum D^T G.
// Reverse, given the adjoints (bars) of the iteration's outputs:
//   latent: Gbar = D Rbar', inside = |v| < mu,
//           vbar = inside ? -(Gbar + Sigmabar') : Gbar,  Sigmabar = -vbar,  Xbar += sum D^T vbar,
//           mubar = -(Sigmabar' + 2 Gbar) sign(v) where not inside;
//   pixel:  P2bar = Lambda2bar' + 2 U2bar', a2bar = P2bar F^T, w2bar = a2bar - Lambda2bar' - U2bar',
//           Xbar += w2bar, Lambda2bar = -w2bar, D9bbar += a2bar, Fbar += a2^T P2bar;
//           P1bar = Lambda1bar' + 2 U1bar', where sampled a1bar = P1bar M1^T,
//           w1bar = rho a1bar - Lambda1bar' - U1bar', D9abar += a1bar, M1bar += a1^T P1bar,
//           rhobar += a1bar . w1; elsewhere w1bar = U1bar';  BXbar = w1bar, Lambda1bar = -w1bar;
//   X:      Xbar += B^T BXbar, Cbar = A^{-1} Xbar (A is symmetric),
//           U1bar = B Cbar, U2bar = Rbar = Cbar for the previous iteration.
// The clamp's derivative at |v| = mu is taken as 0 (the open interval), so the kink counts as
// outside the dead zone.
// Half-window mode: the kept offsets tau stand for the pairs +-tau.  Sigmabar is kept for the kept
// offsets with the full window's values (the -tau half is its mirror image), so the adjoint sum
// of vbar and the threshold partial sums are counted twice, like the forward adjoint sum.
#pragma once
#include "common.cuh"
#include "k_latent.cuh"
#include "k_objective.cuh"

namespace fuse {

// Latent reverse pass of one iteration.  Layouts as the forward latent pass: X [L_s][H][W],
// omega [|W|][H][W], the state re-indexed by the source pixel m = i - k.  Reads the state
// that entered the iteration (Sin) and the adjoint Rbar (= Cbar of the next iteration); Sb holds
// the adjoint of the state the iteration produced and is overwritten with the adjoint of the state
// that entered it.  The adjoint sum sum D^T vbar is written as planes A/V exactly as the forward
// pass writes R (plane tau1 + S: A, plane (2S+1) + tau1 + S: V), and
// part[block] += (half ? 2 : 1) sum mubar * omega(i) over the block's entries.
// Threads: (W/VEC) x Ty rounded up to whole warps (for the block sum), each owning VEC consecutive
// pixels; grid (ceil(H/Ty), L_s, rows of W).
template <typename T, typename WT, int K, int VEC>
__global__ void __launch_bounds__(256)
latent_bwd_kernel(const T* __restrict__ X, const WT* __restrict__ omega, const T* __restrict__ Sin,
                  T* __restrict__ Sb, const T* __restrict__ Rb, T* __restrict__ planes, double* __restrict__ part,
                  int H, int W, int Ls, int S, int Ty, T coef, int half) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Hs = reinterpret_cast<T*>(smem_raw);           // [(2S+1)][Ty][W]
    constexpr int PS = 2 * K + 1;
    constexpr int NP = PS * PS;
    const int tpr = W / VEC;
    const int tid = threadIdx.x;
    const int r = tid / tpr;
    const int x0 = (tid - r * tpr) * VEC;
    const int y = blockIdx.x * Ty + r;
    const TauMap tm{S, half};
    const int t1 = tm.t1_of_block(blockIdx.z);
    const int nt2 = tm.nt2(t1);
    const int c = blockIdx.y;
    const bool valid = r < Ty;                        // the block is rounded up to whole warps
    const bool active = valid && y < H;
    const size_t n = (size_t)H * W;
    const int side = 2 * S + 1;
    const T* Xc = X + (size_t)c * n;
    const T* Rc = Rb + (size_t)c * n;
    const size_t vstride = (size_t)Ls * n / VEC;
    T Xm[VEC], Rm[VEC], A[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        Xm[j] = active ? Xc[(size_t)y * W + x0 + j] : T(0);
        Rm[j] = active ? Rc[(size_t)y * W + x0 + j] : T(0);
        A[j] = T(0);
    }
    double smu = 0.0;                                 // FP64 only across offsets (few adds)
    for (int jt = 0; jt < nt2; ++jt) {
        const int t2 = tm.t2_of(t1, jt);
        T smu_t = T(0);
        T Hacc[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) Hacc[j] = T(0);
        if (active) {
            const int ys = wrap1(y - t1, H);
            T delta[VEC], gb[VEC];
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                const size_t q = (size_t)ys * W + wrap1(x0 + j - t2, W);
                delta[j] = Xm[j] - Xc[q];               // D X at the re-indexed pixel
                gb[j] = Rm[j] - Rc[q];                  // Gbar = D Rbar
            }
            const WT* om = omega + (size_t)tm.w_index(t1, t2) * n;
            const size_t base = ((size_t)tm.s_index(t1, t2) * NP * Ls + c) * n + (size_t)y * W + x0;
            const vecT<T, VEC>* si = reinterpret_cast<const vecT<T, VEC>*>(Sin + base);
            vecT<T, VEC>* sb = reinterpret_cast<vecT<T, VEC>*>(Sb + base);
#pragma unroll
            for (int k1 = -K; k1 <= K; ++k1) {
                const int yw = wrap1(y + k1, H);
                T w[VEC + 2 * K];
#pragma unroll
                for (int j = 0; j < VEC + 2 * K; ++j) w[j] = (T)wload(om + (size_t)yw * W + wrap1(x0 - K + j, W));
                // issue the 2(2K+1) state loads of this patch row before any arithmetic or store
                vecT<T, VEC> s_in[PS], s_b[PS];
                const size_t row0 = (size_t)((k1 + K) * PS) * vstride;
#pragma unroll
                for (int k2 = 0; k2 < PS; ++k2) {
                    s_in[k2] = ld_stream(si + row0 + (size_t)k2 * vstride);
                    s_b[k2] = ld_stream(sb + row0 + (size_t)k2 * vstride);
                }
#pragma unroll
                for (int k2 = 0; k2 < PS; ++k2) {
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        const T v = delta[j] - s_in[k2].v[j];
                        const T wt = w[j + k2];
                        const bool inside = (v < T(0) ? -v : v) < coef * wt;
                        const T vb = inside ? -(gb[j] + s_b[k2].v[j]) : gb[j];
                        if (!inside && v != T(0)) {
                            const T mb = -(s_b[k2].v[j] + T(2) * gb[j]);
                            smu_t += v > T(0) ? mb * wt : -mb * wt;
                        }
                        Hacc[j] += vb;
                        s_b[k2].v[j] = -vb;
                    }
                    st_stream(sb + row0 + (size_t)k2 * vstride, s_b[k2]);
                }
            }
            smu += (double)smu_t;
        }
        if (valid) {
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                A[j] += Hacc[j];
                Hs[((size_t)(t2 + S) * Ty + r) * W + x0 + j] = Hacc[j];
            }
        }
    }
    double v1[1] = {half ? 2.0 * smu : smu};
    block_sum<1, true>(v1, part + ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
    __syncthreads();
    if (!active) return;
    T V[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) V[j] = T(0);
    for (int jt = 0; jt < nt2; ++jt) {
        const int t2 = tm.t2_of(t1, jt);
        const T* hrow = Hs + ((size_t)(t2 + S) * Ty + r) * W;
#pragma unroll
        for (int j = 0; j < VEC; ++j) V[j] += hrow[wrap1(x0 + j + t2, W)];
    }
    vstore<T, VEC>(planes + ((size_t)c * 2 * side + (t1 + S)) * n + (size_t)y * W + x0, A);
    vstore<T, VEC>(planes + ((size_t)c * 2 * side + side + (t1 + S)) * n + (size_t)y * W + x0, V);
}

// Pipelined form of latent_bwd_kernel (same arithmetic, same outputs): the taped state Sin and the
// state adjoint Sb stream through a shared-memory ring of D slots by bulk asynchronous copies
// issued by one producer warp; a slot holds the block's rows of one (tau, k) plane of both.  The
// consumers rewrite Sb in place with streaming stores.  The threshold partials are reduced among
// the consumer warps through shared memory in a fixed order (deterministic) and added to
// part[block].  Every barrier wait is bounded (`limit` polls); a timeout sets bit 1 of *err and
// the block still finishes in bounded time.
template <typename T, typename WT>
struct LatentBwdArgs {
    const T* X;
    const WT* omega;
    const T* Sin;
    T* Sb;
    const T* Rb;
    T* planes;
    double* part;
    int H, W, Ls, S, Ty, ncons, D;
    T coef;
    int* err;
    unsigned limit;
    int half;
};

template <typename T, typename WT, int K, int VEC>
__global__ void __launch_bounds__(288, 2) latent_bwd_tma_kernel(LatentBwdArgs<T, WT> a) {
    extern __shared__ __align__(128) unsigned char smem_tma[];
    constexpr int PS = 2 * K + 1;
    constexpr int NP = PS * PS;
    const int H = a.H, W = a.W, Ls = a.Ls, S = a.S, Ty = a.Ty, ncons = a.ncons, D = a.D;
    const int side = 2 * S + 1;
    const int tile = Ty * W;
    T* ring = reinterpret_cast<T*>(smem_tma);                 // [D][2][Ty][W]: Sin, Sb
    T* Hs = ring + (size_t)D * 2 * tile;                      // [(2S+1)][Ty][W]
    uint64_t* full = reinterpret_cast<uint64_t*>(Hs + (size_t)side * tile);
    uint64_t* empty = full + D;
    __shared__ volatile int s_abort;
    __shared__ double red[9];

    const int tid = threadIdx.x;
    const int tpr = W / VEC;
    const int y0 = blockIdx.x * Ty;
    const int rows = min(Ty, H - y0);
    const TauMap tm{a.S, a.half};
    const int t1 = tm.t1_of_block(blockIdx.z);
    const int nt2 = tm.nt2(t1);
    const int c = blockIdx.y;
    const size_t n = (size_t)H * W;
    const int nq = nt2 * NP;
    const unsigned bytes = (unsigned)(rows * W * (int)sizeof(T));

    if (tid == 0) {
        for (int q = 0; q < D; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], (unsigned)(ncons / 32));
        }
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();

    if (tid >= ncons) {
        // ---------------- producer warp ----------------
        if (tid == ncons) {
            const uint64_t pol = l2_evict_first_policy();
            int issued = 0;
            for (int q = 0; q < nq; ++q) {
                if (s_abort) break;
                const int slot = q % D;
                if (q >= D && !mbar_wait(&empty[slot], (unsigned)((q / D - 1) & 1), a.limit, a.err, 1)) {
                    s_abort = 1;
                    break;
                }
                const int j = q / NP, kidx = q - j * NP;
                const int t2 = tm.t2_of(t1, j);
                const size_t off = ((size_t)(tm.s_index(t1, t2) * NP + kidx) * Ls + c) * n + (size_t)y0 * W;
                mbar_arrive_expect_tx(&full[slot], 2 * bytes);
                tma_load_1d(ring + (size_t)slot * 2 * tile, a.Sin + off, bytes, &full[slot], pol);
                tma_load_1d(ring + (size_t)slot * 2 * tile + tile, a.Sb + off, bytes, &full[slot], pol);
                issued = q + 1;
            }
            const unsigned dlim = a.limit > (1u << 20) ? a.limit : (1u << 20);
            for (int q = issued > D ? issued - D : 0; q < issued; ++q)
                if (!mbar_wait(&full[q % D], (unsigned)((q / D) & 1), dlim, a.err, 1)) break;
        }
        return;
    }

    // ---------------- consumers ----------------
    const int lane = tid & 31;
    const int r = tid / tpr;
    const int x0 = (tid - r * tpr) * VEC;
    const int y = y0 + r;
    const bool owner = tid < tpr * Ty;
    const bool active = owner && r < rows;
    const T* Xc = a.X + (size_t)c * n;
    const T* Rc = a.Rb + (size_t)c * n;
    const size_t pix = (size_t)y * W + x0;
    const size_t xsrow = (size_t)wrap1(y - t1, H) * W;
    const size_t kstride = (size_t)Ls * n;
    T Xm[VEC], Rm[VEC];
    if (active) {
        vload<T, VEC>(Xc + pix, Xm);
        vload<T, VEC>(Rc + pix, Rm);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) { Xm[j] = T(0); Rm[j] = T(0); }
    }
    int slot = 0;
    unsigned par = 0;
    double smu = 0.0;
    for (int jt = 0; jt < nt2; ++jt) {
        const int t2 = tm.t2_of(t1, jt);
        T Hacc[VEC], delta[VEC], gb[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            Hacc[j] = T(0);
            const size_t q = xsrow + wrap1(x0 + j - t2, W);
            delta[j] = active ? Xm[j] - Xc[q] : T(0);           // D X at the re-indexed pixel
            gb[j] = active ? Rm[j] - Rc[q] : T(0);              // Gbar = D Rbar
        }
        const WT* om = a.omega + (size_t)tm.w_index(t1, t2) * n;
        T* gp = a.Sb + ((size_t)tm.s_index(t1, t2) * NP * Ls + c) * n + pix;
        T smu_t = T(0);
#pragma unroll
        for (int k1 = 0; k1 < PS; ++k1) {
            const WT* orow = om + (size_t)wrap1(y + k1 - K, H) * W;
            T w[VEC + 2 * K];
#pragma unroll
            for (int j = 0; j < VEC + 2 * K; ++j) w[j] = active ? (T)wload(orow + wrap1(x0 - K + j, W)) : T(0);
#pragma unroll
            for (int k2 = 0; k2 < PS; ++k2) {
                const unsigned lim = s_abort ? 64u : a.limit;
                if (!mbar_wait(&full[slot], par, lim, a.err, 1)) s_abort = 1;
                if (active) {
                    T sin[VEC], sbv[VEC];
                    const T* rs = ring + (size_t)slot * 2 * tile + (size_t)r * W + x0;
                    vload<T, VEC>(rs, sin);
                    vload<T, VEC>(rs + tile, sbv);
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        const T v = delta[j] - sin[j];
                        const T wt = w[j + k2];
                        const bool inside = (v < T(0) ? -v : v) < a.coef * wt;
                        const T vb = inside ? -(gb[j] + sbv[j]) : gb[j];
                        if (!inside && v != T(0)) {
                            const T mb = -(sbv[j] + T(2) * gb[j]);
                            smu_t += v > T(0) ? mb * wt : -mb * wt;
                        }
                        Hacc[j] += vb;
                        sbv[j] = -vb;
                    }
                    vstore_stream<T, VEC>(gp, sbv);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                gp += kstride;
                if (++slot == D) { slot = 0; par ^= 1u; }
            }
        }
        smu += (double)smu_t;
        if (owner) {
#pragma unroll
            for (int j = 0; j < VEC; ++j) Hs[((size_t)(t2 + S) * Ty + r) * W + x0 + j] = Hacc[j];
        }
    }
    // threshold partials: consumer warps only, fixed order
    const double ws = warp_sum(smu);
    if (lane == 0) red[tid >> 5] = ws;
    consumer_barrier(ncons);                 // every H_tau is in Hs and every warp sum in red
    if (tid == 0) {
        double sum = 0.0;
        for (int q = 0; q < ncons / 32; ++q) sum += red[q];
        double* pp = a.part + ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        *pp += a.half ? 2.0 * sum : sum;
    }
    if (active) {
        T A[VEC], V[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) { A[j] = T(0); V[j] = T(0); }
        for (int jt = 0; jt < nt2; ++jt) {
            const int t2 = tm.t2_of(t1, jt);
            const T* hrow = Hs + ((size_t)(t2 + S) * Ty + r) * W;
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                A[j] += hrow[x0 + j];
                V[j] += hrow[wrap1(x0 + j + t2, W)];
            }
        }
        vstore<T, VEC>(a.planes + ((size_t)c * 2 * side + (t1 + S)) * n + pix, A);
        vstore<T, VEC>(a.planes + ((size_t)c * 2 * side + side + (t1 + S)) * n + pix, V);
    }
}

// Pixel reverse pass of one iteration.
template <typename T>
struct PixelBwdArgs {
    const T* X;        // X of the iteration
    const T* BX;       // B X
    const T* Lam1;     // Lambda1, Lambda2 that entered the iteration
    const T* Lam2;
    const T* U1b;      // adjoints of U1', U2' (= B Cbar, Cbar of the next iteration)
    const T* U2b;
    T* L1b;            // in: adjoints of Lambda1', Lambda2'; out: adjoints of Lambda1, Lambda2
    T* L2b;
    T* Xp;             // out: w2bar (the pixel pass's part of Xbar)
    T* BXb;            // out: w1bar (the adjoint of B X)
    T* D9ab;           // += a1bar on the sampled lattice [L_s][H/d][W/d]
    T* D9bb;           // += a2bar
    const T* D9a;
    const T* D9b;
    const T* M1;       // (E E^T + rho I)^{-1}, row-major
    const T* F;        // (I + lambda1/rho E R R^T E^T)^{-1}, row-major
    const T* Krho;     // d F / d rho, d F / d lambda1, d M1 / d rho (row-major)
    const T* Klam;
    const T* Kmu;
    double* part;      // [blocks][3] += see pixel_bwd_kernel
    int H, W, Ls, d;
    T rho;
    const uint8_t* mask;   // sampling mask [H][W] (d = 1) or NULL for the lattice of ratio d
};

// One thread per pixel, band vectors in registers (MAXLS >= L_s).  Per block, part[3 b + q] +=
//   q = 0: a2 Krho P2bar^T + a1 Kmu P1bar^T + a1bar . w1     (the rho partials of F, M1 and a1)
//   q = 1: a2 Klam P2bar^T                                     (the lambda1 partial of F)
//   q = 2: a2bar . D9b                                         (the rho and lambda1 partials of D9b)
template <typename T, int MAXLS>
__global__ void __launch_bounds__(128) pixel_bwd_kernel(PixelBwdArgs<T> g) {
    const int H = g.H, W = g.W, Ls = g.Ls, d = g.d;
    // the five L_s x L_s matrices, read uniformly by the warp, staged in shared memory
    __shared__ T sm[5][MAXLS * MAXLS];
    for (int i = threadIdx.x; i < Ls * Ls; i += blockDim.x) {
        sm[0][i] = g.F[i];
        sm[1][i] = g.Krho[i];
        sm[2][i] = g.Klam[i];
        sm[3][i] = g.M1[i];
        sm[4][i] = g.Kmu[i];
    }
    __syncthreads();
    const T* __restrict__ sF = sm[0];
    const T* __restrict__ sKr = sm[1];
    const T* __restrict__ sKl = sm[2];
    const T* __restrict__ sM1 = sm[3];
    const T* __restrict__ sKm = sm[4];
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double q[3] = {0.0, 0.0, 0.0};
    if (p < n) {
        T q0 = T(0), q1 = T(0), q2 = T(0);            // per pixel in T, FP64 across pixels
        T pb[MAXLS], a[MAXLS], wb[MAXLS];
        // inputs of the P1 half, read before any store so that every load of the pixel is in
        // flight at once (the stores below may alias them as far as the compiler knows); kept
        // in registers only for the smaller band counts
        constexpr bool kHoist = MAXLS <= 20;
        T pb1[kHoist ? MAXLS : 1], wb1[kHoist ? MAXLS : 1], a1w[kHoist ? MAXLS : 1];
#pragma unroll
        for (int j = 0; j < MAXLS; ++j) {
            if (j < Ls) {
                const T l2b = g.L2b[(size_t)j * n + p], u2b = g.U2b[(size_t)j * n + p];
                pb[j] = l2b + T(2) * u2b;
                wb[j] = -(l2b + u2b);
                a[j] = g.X[(size_t)j * n + p] - g.Lam2[(size_t)j * n + p] + g.D9b[(size_t)j * n + p];
                if constexpr (kHoist) {
                    const T l1b = g.L1b[(size_t)j * n + p], u1b = g.U1b[(size_t)j * n + p];
                    pb1[j] = l1b + T(2) * u1b;
                    wb1[j] = -(l1b + u1b);
                    a1w[j] = g.BX[(size_t)j * n + p] - g.Lam1[(size_t)j * n + p];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < MAXLS; ++i) {
            if (i < Ls) {
                T ab = T(0), kr = T(0), kl = T(0);
#pragma unroll
                for (int j = 0; j < MAXLS; ++j) {
                    if (j < Ls) {
                        ab += pb[j] * sF[i * Ls + j];
                        kr += sKr[i * Ls + j] * pb[j];
                        kl += sKl[i * Ls + j] * pb[j];
                    }
                }
                const T d9b = g.D9b[(size_t)i * n + p];
                q0 += a[i] * kr;
                q1 += a[i] * kl;
                q2 += ab * d9b;
                const T w2b = wb[i] + ab;
                g.Xp[(size_t)i * n + p] = w2b;
                g.L2b[(size_t)i * n + p] = -w2b;
                g.D9bb[(size_t)i * n + p] += ab;
            }
        }
        const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
#pragma unroll
        for (int j = 0; j < MAXLS; ++j) {
            if (j < Ls) {
                if constexpr (kHoist) {
                    pb[j] = pb1[j];
                    wb[j] = wb1[j];
                    a[j] = a1w[j];                                              // w1
                } else {
                    const T l1b = g.L1b[(size_t)j * n + p], u1b = g.U1b[(size_t)j * n + p];
                    pb[j] = l1b + T(2) * u1b;
                    wb[j] = -(l1b + u1b);
                    a[j] = g.BX[(size_t)j * n + p] - g.Lam1[(size_t)j * n + p];  // w1
                }
            }
        }
        if (sampled_pixel(g.mask, p, y, x, d)) {
            const size_t nl = (size_t)(H / d) * (W / d);
            const size_t pl = (size_t)(y / d) * (W / d) + x / d;
#pragma unroll
            for (int i = 0; i < MAXLS; ++i) {
                if (i < Ls) {
                    T ab = T(0), km = T(0);
#pragma unroll
                    for (int j = 0; j < MAXLS; ++j) {
                        if (j < Ls) {
                            ab += pb[j] * sM1[i * Ls + j];
                            km += sKm[i * Ls + j] * pb[j];
                        }
                    }
                    const T a1 = g.rho * a[i] + g.D9a[(size_t)i * nl + pl];
                    q0 += a1 * km + ab * a[i];
                    const T w1b = wb[i] + g.rho * ab;
                    g.BXb[(size_t)i * n + p] = w1b;
                    g.L1b[(size_t)i * n + p] = -w1b;
                    g.D9ab[(size_t)i * nl + pl] += ab;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < MAXLS; ++i) {
                if (i < Ls) {
                    const T w1b = wb[i] + pb[i];             // = U1bar'
                    g.BXb[(size_t)i * n + p] = w1b;
                    g.L1b[(size_t)i * n + p] = -w1b;
                }
            }
        }
        q[0] = (double)q0;
        q[1] = (double)q1;
        q[2] = (double)q2;
    }
    block_sum<3, true>(q, g.part + (size_t)blockIdx.x * 3);
}

// y += x over n elements.
template <typename T>
__global__ void __launch_bounds__(256) axpy_kernel(T* __restrict__ y, const T* __restrict__ x, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

// Kept offset q (the state's offset index) -> (tau1, tau2): inverse of TauMap::s_index.
__device__ __forceinline__ void tau_of_state_index(int q, int S, int half, int* t1, int* t2) {
    const int side = 2 * S + 1;
    if (half) {
        if (q < S) { *t1 = 0; *t2 = q + 1; return; }
        const int r = q - S;
        *t1 = r / side + 1;
        *t2 = r % side - S;
        return;
    }
    const int cell = q >= (side * side) / 2 ? q + 1 : q;
    *t1 = cell / side - S;
    *t2 = cell % side - S;
}

// dL/domega of one reverse iteration, run before the latent reverse pass overwrites the state
// adjoint.  mu = coef omega with coef = lambda2/rho, so for the output pixel i and offset tau
//   omega_bar_tau(i) += scale sum_{k, c} mubar_{tau k c}(i),  scale = coef (x2 in half-window mode:
//   the stored weight of a kept offset also thresholds its mirror),
//   mubar = -(Sigmabar' + 2 Gbar) sign(v) outside the dead zone, 0 inside,
// with v, Gbar as in the latent reverse pass, read at the re-indexed pixel m = i - k.
// One thread per output pixel (coalesced over m for every (k, c)); grid (ceil(n/256), kept offsets).
template <typename T, typename WT, int K>
__global__ void __launch_bounds__(256)
omega_bwd_kernel(const T* __restrict__ X, const WT* __restrict__ omega, const T* __restrict__ Sin,
                 const T* __restrict__ Sb, const T* __restrict__ Rb, T* __restrict__ omega_bar,
                 int H, int W, int Ls, int S, T coef, T scale, int half) {
    constexpr int PS = 2 * K + 1;
    constexpr int NP = PS * PS;
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int q = blockIdx.y;
    int t1, t2;
    tau_of_state_index(q, S, half, &t1, &t2);
    const TauMap tm{S, half};
    const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
    const int wi = tm.w_index(t1, t2);
    const T mu = coef * (T)wload(omega + (size_t)wi * n + p);
    T acc = T(0);
#pragma unroll
    for (int k1 = -K; k1 <= K; ++k1) {
        const int my = wrapn(y - k1, H);
        const int sy = wrapn(my - t1, H);
#pragma unroll
        for (int k2 = -K; k2 <= K; ++k2) {
            const int mx = wrapn(x - k2, W);
            const int sx = wrapn(mx - t2, W);
            const size_t m = (size_t)my * W + mx, ms = (size_t)sy * W + sx;
            const size_t base = ((size_t)q * NP + (k1 + K) * PS + (k2 + K)) * Ls * n + m;
            for (int c = 0; c < Ls; ++c) {
                const size_t cn = (size_t)c * n;
                const T v = X[cn + m] - X[cn + ms] - Sin[base + cn];
                if ((v < T(0) ? -v : v) < mu || v == T(0)) continue;
                const T mb = -(Sb[base + cn] + T(2) * (Rb[cn + m] - Rb[cn + ms]));
                acc += v > T(0) ? mb : -mb;
            }
        }
    }
    omega_bar[(size_t)wi * n + p] += scale * acc;
}

// Guide gradient through the weights (eq. wts), step 1: for every stored offset tau
//   A_tau(m) = sum_{k in [-K,K]^2} a_tau(m + k),  a_tau = c2 omega_bar_tau omega_tau, c2 = -2/h^2.
// One thread per pixel; grid (ceil(n/256), |W|).
template <typename T, typename WT>
__global__ void __launch_bounds__(256)
guide_box_kernel(const T* __restrict__ omega_bar, const WT* __restrict__ omega, T* __restrict__ A,
                 int H, int W, int K, T c2) {
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const size_t off = (size_t)blockIdx.y * n;
    const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
    T acc = T(0);
    for (int k1 = -K; k1 <= K; ++k1) {
        const size_t row = (size_t)wrapn(y + k1, H) * W;
        for (int k2 = -K; k2 <= K; ++k2) {
            const size_t j = row + wrapn(x + k2, W);
            acc += omega_bar[off + j] * (T)wload(omega + off + j);
        }
    }
    A[off + p] = c2 * acc;
}

// Step 2: dL/dG_c(j) = sum_tau [A_tau(j) (G_c(j) - G_c(j - tau)) - A_tau(j + tau) (G_c(j + tau) - G_c(j))]
// (the adjoint of the patch differences D_{tau k} G summed over k).  One thread per pixel;
// grid (ceil(n/256), L_guide).
template <typename T>
__global__ void __launch_bounds__(256)
guide_bwd_kernel(const T* __restrict__ G, const T* __restrict__ A, T* __restrict__ Gb, int H, int W, int S) {
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int side = 2 * S + 1;
    const int nW = side * side - 1;
    const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
    const T* Gc = G + (size_t)blockIdx.y * n;
    const T g0 = Gc[p];
    T acc = T(0);
    for (int t = 0; t < nW; ++t) {
        const int cell = t >= nW / 2 ? t + 1 : t;
        const int t1 = cell / side - S, t2 = cell % side - S;
        const size_t jm = (size_t)wrapn(y - t1, H) * W + wrapn(x - t2, W);
        const size_t jp = (size_t)wrapn(y + t1, H) * W + wrapn(x + t2, W);
        const T* At = A + (size_t)t * n;
        acc += At[p] * (g0 - Gc[jm]) - At[jp] * (Gc[jp] - g0);
    }
    Gb[(size_t)blockIdx.y * n + p] = acc;
}

}  // namespace fuse
