// 2D DFT solve of the X system (Sec. IV-A eqs. x_linear_system_main and inv):
//   X_c = IDFT( f(w) * DFT(C_c) ),  f(w) = 1 / (1 + |b^(w)|^2 + |P| sum_tau |d^_{tau 0}(w)|^2),
// f real and even, precomputed in FP64 on the host and pre-scaled by 1/(H W).
//
// Two real bands ride in one complex transform, z = C_{2p} + i C_{2p+1}: since f is real and
// even, filtering z returns X_{2p} + i X_{2p+1}.  Three passes over [L_s/2][H][W] complex:
//   rows forward (loads the real pairs), columns forward * f * columns inverse (one kernel),
//   rows inverse (stores the real pairs).
// Each 1D transform runs in shared memory as a self-sorting (Stockham) mixed-radix FFT
// with radices 4, 2, 3, 5: at a stage of radix r with Ns points already combined, butterfly
// j reads in[j + m N/r] (m < r), twists them by w^{m (j mod Ns) N/(Ns r)} with
// w = exp(-2 pi i / N) (conjugated for the inverse), does an r-point DFT and writes
// out[(j div Ns) Ns r + (j mod Ns) + q Ns] (q < r).  Twiddles come from a table computed on
// the host in FP64.
#pragma once
#include "common.cuh"

namespace fuse {

struct FFTPlan {
    int N;
    int nst;
    int rad[20];
};

template <typename T, int R>
__device__ __forceinline__ void small_dft(cplx<T>* v, int sign, const cplx<T>* __restrict__ tw, int N) {
    if constexpr (R == 2) {
        cplx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        cplx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        cplx<T> c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        cplx<T> id = {-d.y, d.x};                       // i * d
        if (sign < 0) { id.x = -id.x; id.y = -id.y; }   // sign * i * d
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, id);
        v[3] = csub(b, id);
    } else {
        cplx<T> in[R];
#pragma unroll
        for (int m = 0; m < R; ++m) in[m] = v[m];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            cplx<T> acc = in[0];
#pragma unroll
            for (int m = 1; m < R; ++m) {
                cplx<T> w = tw[((m * q) % R) * (N / R)];
                if (sign > 0) w.y = -w.y;
                acc = cadd(acc, cmul(in[m], w));
            }
            v[q] = acc;
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* in, cplx<T>* out, int N, int Ns, int sign,
                                          const cplx<T>* __restrict__ tw, int t, int nt) {
    const int Nr = N / R;
    const int step = N / (Ns * R);
    for (int j = t; j < Nr; j += nt) {
        const int kk = j % Ns;
        cplx<T> v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = in[j + m * Nr];
        if (kk) {
#pragma unroll
            for (int m = 1; m < R; ++m) {
                cplx<T> w = tw[m * kk * step];
                if (sign > 0) w.y = -w.y;
                v[m] = cmul(v[m], w);
            }
        }
        small_dft<T, R>(v, sign, tw, N);
        const int base = (j / Ns) * Ns * R + kk;
#pragma unroll
        for (int q = 0; q < R; ++q) out[base + q * Ns] = v[q];
    }
}

// Runs all stages (block-wide barriers between stages); returns the buffer with the result.
template <typename T>
__device__ cplx<T>* fft_smem(cplx<T>* a, cplx<T>* b, const FFTPlan& P, const cplx<T>* __restrict__ tw,
                             int sign, int t, int nt) {
    int Ns = 1;
    for (int s = 0; s < P.nst; ++s) {
        const int r = P.rad[s];
        switch (r) {
            case 4: fft_stage<T, 4>(a, b, P.N, Ns, sign, tw, t, nt); break;
            case 2: fft_stage<T, 2>(a, b, P.N, Ns, sign, tw, t, nt); break;
            case 3: fft_stage<T, 3>(a, b, P.N, Ns, sign, tw, t, nt); break;
            default: fft_stage<T, 5>(a, b, P.N, Ns, sign, tw, t, nt); break;
        }
        __syncthreads();
        cplx<T>* tmp = a; a = b; b = tmp;
        Ns *= r;
    }
    return a;
}

// Rows forward: z(y, .) = C_{2p}(y, .) + i C_{2p+1}(y, .), transformed along x.
// Block: rpb rows x tpr threads; grid (ceil(H/rpb), ceil(L_s/2)).
template <typename T>
__global__ void __launch_bounds__(256)
fft_rows_fwd_kernel(const T* __restrict__ C, cplx<T>* __restrict__ Y, int H, int W, int Ls,
                    FFTPlan P, const cplx<T>* __restrict__ tw, int rpb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int tpr = blockDim.x / rpb;
    const int rr = threadIdx.x / tpr, t = threadIdx.x - rr * tpr;
    const int y = blockIdx.x * rpb + rr;
    const int p = blockIdx.y;
    const size_t n = (size_t)H * W;
    cplx<T>* b0 = sm + (size_t)rr * 2 * W;
    cplx<T>* b1 = b0 + W;
    const bool ok = y < H;
    const T* re = C + (size_t)(2 * p) * n + (size_t)y * W;
    const bool has_im = 2 * p + 1 < Ls;
    const T* im = C + (size_t)(2 * p + 1) * n + (size_t)y * W;
    for (int x = t; x < W; x += tpr) {
        cplx<T> z = {T(0), T(0)};
        if (ok) { z.x = re[x]; if (has_im) z.y = im[x]; }
        b0[x] = z;
    }
    __syncthreads();
    cplx<T>* res = fft_smem(b0, b1, P, tw, -1, t, tpr);
    if (ok)
        for (int x = t; x < W; x += tpr) Y[(size_t)p * n + (size_t)y * W + x] = res[x];
}

// Columns: forward along y, multiply by f(u, v), inverse along y, for CW columns per block.
// Block: CW x tpc threads (warp-major per column); grid (ceil(W/CW), ceil(L_s/2)).
template <typename T>
__global__ void __launch_bounds__(256)
fft_cols_kernel(cplx<T>* __restrict__ Y, const T* __restrict__ f, int H, int W, FFTPlan P,
                const cplx<T>* __restrict__ tw, int CW) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int tpc = blockDim.x / CW;
    const int cw = threadIdx.x / tpc, t = threadIdx.x - cw * tpc;
    const int x0 = blockIdx.x * CW;
    const int p = blockIdx.y;
    const size_t n = (size_t)H * W;
    const int pitch = 2 * H + 1;
    cplx<T>* Yp = Y + (size_t)p * n;
    for (int idx = threadIdx.x; idx < H * CW; idx += blockDim.x) {
        const int row = idx / CW, cc = idx - row * CW;
        const int x = x0 + cc;
        sm[(size_t)cc * pitch + row] = x < W ? Yp[(size_t)row * W + x] : cplx<T>{T(0), T(0)};
    }
    __syncthreads();
    cplx<T>* b0 = sm + (size_t)cw * pitch;
    cplx<T>* b1 = b0 + H;
    cplx<T>* res = fft_smem(b0, b1, P, tw, -1, t, tpc);
    const int x = x0 + cw;
    if (x < W) {
        for (int u = t; u < H; u += tpc) {
            const T g = f[(size_t)u * W + x];
            res[u].x *= g;
            res[u].y *= g;
        }
    }
    __syncthreads();
    cplx<T>* other = res == b0 ? b1 : b0;
    res = fft_smem(res, other, P, tw, +1, t, tpc);
    // the result buffer of column cc sits at the same parity for every column
    const int off = (int)(res - b0);
    for (int idx = threadIdx.x; idx < H * CW; idx += blockDim.x) {
        const int row = idx / CW, cc = idx - row * CW;
        const int xx = x0 + cc;
        if (xx < W) Yp[(size_t)row * W + xx] = sm[(size_t)cc * pitch + off + row];
    }
}

// Rows inverse: X_{2p} = Re, X_{2p+1} = Im of the inverse transform along x (f carries 1/(HW)).
template <typename T>
__global__ void __launch_bounds__(256)
fft_rows_inv_kernel(const cplx<T>* __restrict__ Y, T* __restrict__ X, int H, int W, int Ls,
                    FFTPlan P, const cplx<T>* __restrict__ tw, int rpb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int tpr = blockDim.x / rpb;
    const int rr = threadIdx.x / tpr, t = threadIdx.x - rr * tpr;
    const int y = blockIdx.x * rpb + rr;
    const int p = blockIdx.y;
    const size_t n = (size_t)H * W;
    cplx<T>* b0 = sm + (size_t)rr * 2 * W;
    cplx<T>* b1 = b0 + W;
    const bool ok = y < H;
    for (int x = t; x < W; x += tpr)
        b0[x] = ok ? Y[(size_t)p * n + (size_t)y * W + x] : cplx<T>{T(0), T(0)};
    __syncthreads();
    cplx<T>* res = fft_smem(b0, b1, P, tw, +1, t, tpr);
    if (!ok) return;
    T* re = X + (size_t)(2 * p) * n + (size_t)y * W;
    const bool has_im = 2 * p + 1 < Ls;
    T* im = X + (size_t)(2 * p + 1) * n + (size_t)y * W;
    for (int x = t; x < W; x += tpr) {
        re[x] = res[x].x;
        if (has_im) im[x] = res[x].y;
    }
}

}  // namespace fuse
