// Circular 2D blur stencils (Sec. I-A): out(i) = sum_{u,v} taps(u,v) in(i + (u,v)), with
// taps = b for B^T (correlation) and taps(u,v) = b(-u,-v) for B (convolution).
//
// MODE 0: out = stencil(in)                                        -> B X
// MODE 1: out = stencil(U1) + U2 + R,  R(j) = sum_{tau1} [A_{tau1}(j) - V_{tau1}(j + (tau1,0))]
//         (half-window mode: tau1 >= 0 only and R doubled, see k_latent.cuh)
//         the right-hand side C = B^T(P1 + Lambda1) + P2 + Lambda2 + sum D^T(Q + Sigma)
//         (Sec. IV-A, after eq. x_linear_system_main), with R from the latent pass planes.
// Tiles of 32 x 32 pixels of one band; the halo is loaded with circular wrap.
#pragma once
#include "common.cuh"

namespace fuse {

constexpr int ST_TX = 32, ST_TY = 32, ST_BY = 8;

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
stencil_kernel(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ taps, int bh, int bw,
               int H, int W, const T* __restrict__ U2, const T* __restrict__ planes, int S, int half) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int th = ST_TY + bh - 1, tw = ST_TX + bw - 1;
    T* tile = reinterpret_cast<T*>(smem_raw);        // [th][tw]
    T* tp = tile + (size_t)th * tw;                  // [bh][bw]
    const int rh = bh / 2, rw = bw / 2;
    const int c = blockIdx.z;
    const int x0 = blockIdx.x * ST_TX, y0 = blockIdx.y * ST_TY;
    const size_t n = (size_t)H * W;
    const T* inc = in + (size_t)c * n;
    const int tid = threadIdx.y * ST_TX + threadIdx.x;
    const int nthr = ST_TX * ST_BY;
    for (int idx = tid; idx < th * tw; idx += nthr) {
        const int rr = idx / tw, cc = idx - rr * tw;
        tile[idx] = inc[(size_t)wrapn(y0 - rh + rr, H) * W + wrapn(x0 - rw + cc, W)];
    }
    for (int idx = tid; idx < bh * bw; idx += nthr) tp[idx] = taps[idx];
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    const int side = 2 * S + 1;
#pragma unroll
    for (int q = 0; q < ST_TY / ST_BY; ++q) {
        const int ly = threadIdx.y + q * ST_BY;
        const int y = y0 + ly;
        if (y >= H) break;
        T acc = T(0);
        for (int u = 0; u < bh; ++u) {
            const T* trow = tile + (size_t)(ly + u) * tw + threadIdx.x;
            const T* krow = tp + u * bw;
            for (int v = 0; v < bw; ++v) acc += krow[v] * trow[v];
        }
        const size_t pix = (size_t)y * W + x;
        if constexpr (MODE == 1) {
            const T* pc = planes + (size_t)c * 2 * side * n;
            T rs = T(0);
            for (int t1 = half ? 0 : -S; t1 <= S; ++t1) {
                rs += pc[(size_t)(t1 + S) * n + pix];
                rs -= pc[(size_t)(side + t1 + S) * n + (size_t)wrap1(y + t1, H) * W + x];
            }
            acc += U2[(size_t)c * n + pix] + (half ? T(2) * rs : rs);
        }
        out[(size_t)c * n + pix] = acc;
    }
}

}  // namespace fuse
