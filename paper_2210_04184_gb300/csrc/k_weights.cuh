// Guide weights omega_{i tau} = exp(-||P_{i tau}(G)||_2^2 / h^2)  (Sec. II-B eq. wts).
//
// ||P_{i tau}(G)||^2 = sum_{k in [-K,K]^2} e_tau(i - k) with the per-pixel squared guide
// difference e_tau(j) = sum_c (G_c(j) - G_c(j - tau))^2, i.e. a (2K+1)^2 box sum of e_tau.
// One block owns Ty output rows (full width) of one offset tau: it forms e_tau on the rows
// [y0-K, y0+Ty+K) in shared memory, box-sums along x, then along y, and stores
// exp(-s/h^2) in the weight type (bf16 rounding is round-to-nearest-even).
#pragma once
#include "common.cuh"

namespace fuse {

template <typename T, typename WT>
__global__ void __launch_bounds__(256)
weights_kernel(const T* __restrict__ G, WT* __restrict__ omega, int H, int W, int Lg, int K, int S,
               int Ty, T inv_h2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rows = Ty + 2 * K;
    T* e = reinterpret_cast<T*>(smem_raw);          // [rows][W]
    T* hs = e + (size_t)rows * W;                   // [rows][W]
    const int side = 2 * S + 1;
    const int tidx = blockIdx.y;
    const int cell = tidx >= (side * side) / 2 ? tidx + 1 : tidx;
    const int t1 = cell / side - S, t2 = cell % side - S;
    const int y0 = blockIdx.x * Ty;
    const size_t n = (size_t)H * W;

    for (int idx = threadIdx.x; idx < rows * W; idx += blockDim.x) {
        const int rr = idx / W, x = idx - rr * W;
        const int yy = wrapn(y0 - K + rr, H);
        const int ys = wrapn(yy - t1, H), xs = wrapn(x - t2, W);
        T acc = T(0);
        for (int c = 0; c < Lg; ++c) {
            const T d = G[(size_t)c * n + (size_t)yy * W + x] - G[(size_t)c * n + (size_t)ys * W + xs];
            acc += d * d;
        }
        e[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows * W; idx += blockDim.x) {
        const int rr = idx / W, x = idx - rr * W;
        T acc = T(0);
        for (int k2 = -K; k2 <= K; ++k2) acc += e[rr * W + wrapn(x - k2, W)];
        hs[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < Ty * W; idx += blockDim.x) {
        const int r = idx / W, x = idx - r * W;
        const int y = y0 + r;
        if (y >= H) continue;
        T s = T(0);
        for (int k1 = -K; k1 <= K; ++k1) s += hs[(r + K - k1) * W + x];
        wstore(omega + (size_t)tidx * n + (size_t)y * W + x, texp(-s * inv_h2));
    }
}

}  // namespace fuse
