// Objective of eq. mainoptim at the current X, off the iteration loop:
//   1/2 ||Y_l - S B X E||^2,  lambda1/2 ||Y_h - X E R||^2,  phi(X) (eq. regfilt1), ||X||^2.
// Per-block partial sums in FP64 (warp shuffles), summed on the host.
#pragma once
#include "common.cuh"

namespace fuse {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV values per thread into out[NV] (thread 0 writes; ACC adds to out instead
// of overwriting it).  blockDim % 32 == 0.
template <int NV, bool ACC = false>
__device__ void block_sum(double (&v)[NV], double* out) {
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = warp_sum(v[q]);
        if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = lane < nw ? red[q][lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) out[q] = ACC ? out[q] + s : s;
        }
    }
}

// partial[blockIdx.x * 3 + {0,1,2}] = sums of (Y_l - S B X E)^2, (Y_h - X E R)^2, X^2 (with a
// sampling mask, Y_l is full resolution and only the masked pixels enter).
template <typename T>
__global__ void __launch_bounds__(256)
obj_data_kernel(const T* __restrict__ X, const T* __restrict__ BX, const T* __restrict__ Yl,
                const T* __restrict__ Yh, const double* __restrict__ E, const double* __restrict__ ER,
                int H, int W, int d, int Ls, int Ll, int Lh, double* __restrict__ partial,
                const uint8_t* __restrict__ mask) {
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (p < n) {
        const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
        for (int c = 0; c < Ls; ++c) { const double a = (double)X[c * n + p]; v[2] += a * a; }
        for (int h = 0; h < Lh; ++h) {
            double r = (double)Yh[h * n + p];
            for (int c = 0; c < Ls; ++c) r -= (double)X[c * n + p] * ER[c * Lh + h];
            v[1] += r * r;
        }
        if (sampled_pixel(mask, p, y, x, d)) {
            const size_t nl = (size_t)(H / d) * (W / d);
            const size_t pl = (size_t)(y / d) * (W / d) + x / d;
            for (int l = 0; l < Ll; ++l) {
                double r = (double)Yl[l * nl + pl];
                for (int c = 0; c < Ls; ++c) r -= (double)BX[c * n + p] * E[c * Ll + l];
                v[0] += r * r;
            }
        }
    }
    block_sum<3>(v, partial + (size_t)blockIdx.x * 3);
}

// partial[blockIdx.y * gridDim.x + blockIdx.x] = sum_i omega_tau(i) sum_{k,c} |D_{tau k} X(i,c)|
// for tau = blockIdx.y.
template <typename T, typename WT>
__global__ void __launch_bounds__(256)
obj_phi_kernel(const T* __restrict__ X, const WT* __restrict__ omega, int H, int W, int Ls, int K, int S,
               double* __restrict__ partial) {
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int side = 2 * S + 1;
    const int tidx = blockIdx.y;
    const int cell = tidx >= (side * side) / 2 ? tidx + 1 : tidx;
    const int t1 = cell / side - S, t2 = cell % side - S;
    double v[1] = {0.0};
    if (p < n) {
        const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
        double s = 0.0;
        for (int c = 0; c < Ls; ++c) {
            const T* Xc = X + (size_t)c * n;
            T sc = T(0);
            for (int k1 = -K; k1 <= K; ++k1)
                for (int k2 = -K; k2 <= K; ++k2) {
                    const T a = Xc[(size_t)wrapn(y - k1, H) * W + wrapn(x - k2, W)];
                    const T b = Xc[(size_t)wrapn(y - t1 - k1, H) * W + wrapn(x - t2 - k2, W)];
                    sc += a > b ? a - b : b - a;
                }
            s += (double)sc;
        }
        v[0] = (double)wload(omega + (size_t)tidx * n + p) * s;
    }
    block_sum<1>(v, partial + (size_t)blockIdx.y * gridDim.x + blockIdx.x);
}

}  // namespace fuse
