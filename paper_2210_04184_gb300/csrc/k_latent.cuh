// Fused latent pass of one ADMM iteration: Q update (eq. Qj_main), Sigma dual update
// (eq. dualvar3_main) and the adjoint sum sum_{tau,k} D_{tau k}^T (Q + Sigma) that enters the
// next right-hand side C (Sec. IV-A, after eq. x_linear_system_main).
//
// Exact rewrite used here.  With v = D_{tau k} X - Sigma and mu = lambda2 omega / rho,
//   Q' = S(v, mu) = v - clamp(v, -mu, mu),
//   Sigma' = Sigma - (D_{tau k}X - Q') = -clamp(v, -mu, mu),
//   G = Q' + Sigma' = v - 2 clamp(v, -mu, mu),
// so Q never has to be stored.  The state is kept re-indexed by the source pixel of the
// shift identity D_{tau k}X(i) = D_{tau 0}X(i - k) (Sec. III): Sig'_{tau k}(m) =
// Sigma_{tau k}(m + k).  For a pixel m the pass then needs delta = X(m) - X(m - tau) once
// per tau, the weight omega_tau(m + k) (the threshold is indexed by the output pixel
// i = m + k, eq. regfilt1) and the contiguous stream Sig'_{tau k}(m).
// The adjoint D_{tau k}^T sends +G to pixel i - k = m and -G to m - tau, so with
// H_tau(m) = sum_k G_{tau k}(m + k):
//   R(j) = sum_tau H_tau(j) - sum_tau H_tau(j + tau).
// One block owns rows [y0, y0+Ty) over the full width, one tau1 and one band c, and writes
//   A_{tau1}(m) = sum_{tau2} H_{(tau1,tau2)}(m)          (plane tau1 + S)
//   V_{tau1}(m) = sum_{tau2} H_{(tau1,tau2)}(m + (0,tau2)) (plane (2S+1) + tau1 + S)
// so that R(j) = sum_{tau1} [A_{tau1}(j) - V_{tau1}(j + (tau1, 0))], summed in fixed order by
// the right-hand-side kernel (deterministic, no atomics).
//
// Layouts: X [L_s][H][W]; omega [|W|][H][W]; Sig' [|W|][|P|][L_s][H][W];
// planes [L_s][2(2S+1)][H][W].  Threads: (W/VEC) x Ty, each owning VEC consecutive pixels.
#pragma once
#include "common.cuh"

namespace fuse {

template <typename T, typename WT, int K, int VEC>
__global__ void __launch_bounds__(256)
latent_kernel(const T* __restrict__ X, const WT* __restrict__ omega, T* __restrict__ Sig,
              T* __restrict__ planes, int H, int W, int Ls, int S, int Ty, T coef) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Hs = reinterpret_cast<T*>(smem_raw);           // [(2S+1)][Ty][W]
    constexpr int PS = 2 * K + 1;
    constexpr int NP = PS * PS;
    const int tpr = W / VEC;
    const int tid = threadIdx.x;
    const int r = tid / tpr;
    const int x0 = (tid - r * tpr) * VEC;
    const int y = blockIdx.x * Ty + r;
    const int t1 = (int)blockIdx.y - S;
    const int c = blockIdx.z;
    const bool active = y < H;
    const size_t n = (size_t)H * W;
    const int side = 2 * S + 1;
    const int centre = (side * side) / 2;
    const T* Xc = X + (size_t)c * n;
    const size_t kstride = (size_t)Ls * n;

    T Xm[VEC];
    T A[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) { Xm[j] = active ? Xc[(size_t)y * W + x0 + j] : T(0); A[j] = T(0); }

    for (int t2 = -S; t2 <= S; ++t2) {
        T Hacc[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) Hacc[j] = T(0);
        if (active && (t1 != 0 || t2 != 0)) {
            const int cell = (t1 + S) * side + (t2 + S);
            const int tidx = cell > centre ? cell - 1 : cell;
            const int ys = wrap1(y - t1, H);
            T delta[VEC];
#pragma unroll
            for (int j = 0; j < VEC; ++j) delta[j] = Xm[j] - Xc[(size_t)ys * W + wrap1(x0 + j - t2, W)];
            const WT* om = omega + (size_t)tidx * n;
            vecT<T, VEC>* sp = reinterpret_cast<vecT<T, VEC>*>(
                Sig + ((size_t)tidx * NP * Ls + c) * n + (size_t)y * W + x0);
            const size_t vstride = kstride / VEC;
#pragma unroll
            for (int k1 = -K; k1 <= K; ++k1) {
                // mu for the output pixels i = m + k, k2 in [-K, K]: columns x0-K .. x0+VEC-1+K
                const int yw = wrap1(y + k1, H);
                T mu[VEC + 2 * K];
#pragma unroll
                for (int j = 0; j < VEC + 2 * K; ++j)
                    mu[j] = coef * (T)wload(om + (size_t)yw * W + wrap1(x0 - K + j, W));
                // issue the 2K+1 loads of this patch row before any store
                vecT<T, VEC> s[PS];
#pragma unroll
                for (int k2 = 0; k2 < PS; ++k2) s[k2] = ld_stream(sp + (size_t)k2 * vstride);
#pragma unroll
                for (int k2 = 0; k2 < PS; ++k2) {
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        const T u = s[k2].v[j] - delta[j];         // -v
                        const T m = mu[j + k2];
                        const T s2 = tmin(tmax(u, -m), m);         // Sigma' = -clamp(v)
                        Hacc[j] += T(2) * s2 - u;                  // G = v + 2 Sigma'
                        s[k2].v[j] = s2;
                    }
                    st_stream(sp + (size_t)k2 * vstride, s[k2]);
                }
                sp += (size_t)PS * vstride;
            }
        }
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            A[j] += Hacc[j];
            Hs[((size_t)(t2 + S) * Ty + r) * W + x0 + j] = Hacc[j];
        }
    }
    __syncthreads();
    if (!active) return;
    T V[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) V[j] = T(0);
    for (int t2 = -S; t2 <= S; ++t2) {
        const T* row = Hs + ((size_t)(t2 + S) * Ty + r) * W;
#pragma unroll
        for (int j = 0; j < VEC; ++j) V[j] += row[wrap1(x0 + j + t2, W)];
    }
    T* pa = planes + ((size_t)c * 2 * side + (t1 + S)) * n + (size_t)y * W + x0;
    T* pv = planes + ((size_t)c * 2 * side + side + (t1 + S)) * n + (size_t)y * W + x0;
    vecT<T, VEC> va, vv;
#pragma unroll
    for (int j = 0; j < VEC; ++j) { va.v[j] = A[j]; vv.v[j] = V[j]; }
    *reinterpret_cast<vecT<T, VEC>*>(pa) = va;
    *reinterpret_cast<vecT<T, VEC>*>(pv) = vv;
}

}  // namespace fuse
