// Per-pixel closed forms of Sec. IV (one thread per pixel, all L_s bands):
//   P2 = (X - Lambda2 + lambda1/rho Y_h R^T E^T) F                       (eq. Qm_update)
//   P1 = S^T S (rho B X + S^T Y_l E^T - rho Lambda1)(E E^T + rho I)^{-1}
//        + (I - S^T S)(B X - Lambda1)                                   (eq. Qh_update)
//   Lambda1 <- Lambda1 - (B X - P1),  Lambda2 <- Lambda2 - (X - P2)      (eqs. dualvar1_main, 2)
// and writes U1 = P1 + Lambda1, U2 = P2 + Lambda2 for the next right-hand side.
// S^T S is the 0/1 mask of pixels with i1 = i2 = 0 (mod d); S^T Y_l E^T at those pixels is
// D9a[c][i1/d][i2/d]; lambda1/rho Y_h R^T E^T is D9b[c][i1][i2].
#pragma once
#include "common.cuh"

namespace fuse {

// One thread per pixel; the pixel's band vectors live in registers (MAXLS >= L_s, loops unrolled
// with guards so the arrays are indexed statically), every input band is loaded once, and the
// L_s x L_s matrices sit in shared memory and are read uniformly by the warp.
template <typename T>
struct PixelArgs {
    const T* X;
    const T* BX;
    T* Lam1;
    T* U1;
    T* Lam2;
    T* U2;
    const T* D9a;
    const T* D9b;
    const T* M1;
    const T* F;
    int H, W, Ls, d;
    T rho;
    const uint8_t* mask;   // sampling mask [H][W] (d = 1) or NULL for the lattice of ratio d
    int no_p1;             // 1: P2 and Lambda2 only (the variant with S B in the X system has no P1)
};

template <typename T, int MAXLS>
__device__ __forceinline__ void pixel_body(const PixelArgs<T>& args, int bx, unsigned char* smem_raw) {
    const T* __restrict__ X = args.X;
    const T* __restrict__ BX = args.BX;
    T* __restrict__ Lam1 = args.Lam1;
    T* __restrict__ U1 = args.U1;
    T* __restrict__ Lam2 = args.Lam2;
    T* __restrict__ U2 = args.U2;
    const T* __restrict__ D9a = args.D9a;
    const T* __restrict__ D9b = args.D9b;
    const int H = args.H, W = args.W, Ls = args.Ls, d = args.d;
    const T rho = args.rho;
    T* sF = reinterpret_cast<T*>(smem_raw);              // [Ls][Ls]
    T* sM = sF + (size_t)Ls * Ls;                        // [Ls][Ls]
    const int tid = threadIdx.x, nb = blockDim.x;
    for (int i = tid; i < Ls * Ls; i += nb) { sF[i] = args.F[i]; sM[i] = args.M1[i]; }
    __syncthreads();
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)bx * nb + tid;
    if (p >= n) return;
    T a[MAXLS], w[MAXLS], w1[MAXLS];
    const bool p1 = !args.no_p1;
    // P2 and Lambda2: a = X - Lambda2 + lambda1/rho Y_h R^T E^T, w = X - Lambda2; the P1 side's
    // w1 = B X - Lambda1 is read here too, before any store, so all loads of the pixel are in flight
#pragma unroll
    for (int j = 0; j < MAXLS; ++j) {
        if (j < Ls) {
            w[j] = X[(size_t)j * n + p] - Lam2[(size_t)j * n + p];
            a[j] = w[j] + D9b[(size_t)j * n + p];
            w1[j] = p1 ? BX[(size_t)j * n + p] - Lam1[(size_t)j * n + p] : T(0);
        }
    }
#pragma unroll
    for (int c = 0; c < MAXLS; ++c) {
        if (c < Ls) {
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < MAXLS; ++j)
                if (j < Ls) acc += a[j] * sF[j * Ls + c];
            const T l2 = acc - w[c];
            Lam2[(size_t)c * n + p] = l2;
            U2[(size_t)c * n + p] = acc + l2;
        }
    }
    if (!p1) return;
    // P1 and Lambda1: w = B X - Lambda1
#pragma unroll
    for (int j = 0; j < MAXLS; ++j)
        if (j < Ls) w[j] = w1[j];
    const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
    if (sampled_pixel(args.mask, p, y, x, d)) {
        const size_t nl = (size_t)(H / d) * (W / d);
        const size_t pl = (size_t)(y / d) * (W / d) + x / d;
#pragma unroll
        for (int j = 0; j < MAXLS; ++j)
            if (j < Ls) a[j] = rho * w[j] + D9a[(size_t)j * nl + pl];
#pragma unroll
        for (int c = 0; c < MAXLS; ++c) {
            if (c < Ls) {
                T acc = T(0);
#pragma unroll
                for (int j = 0; j < MAXLS; ++j)
                    if (j < Ls) acc += a[j] * sM[j * Ls + c];
                const T l1 = acc - w[c];
                Lam1[(size_t)c * n + p] = l1;
                U1[(size_t)c * n + p] = acc + l1;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < MAXLS; ++c) {
            if (c < Ls) {                                    // P1 = B X - Lambda1, Lambda1 = 0
                Lam1[(size_t)c * n + p] = T(0);
                U1[(size_t)c * n + p] = w[c];
            }
        }
    }
}

template <typename T, int MAXLS>
__global__ void __launch_bounds__(128) pixel_kernel(PixelArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pixel_body<T, MAXLS>(a, blockIdx.x, smem_raw);
}

template <typename T, int MAXLS>
__global__ void __launch_bounds__(128)
pixel_batch_kernel(const PixelArgs<T>* __restrict__ args, const Segment* __restrict__ seg, int nseg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int prob, bx, by, bz;
    segment_of_block(seg, nseg, blockIdx.x, &prob, &bx, &by, &bz);
    const PixelArgs<T> a = args[prob];
    pixel_body<T, MAXLS>(a, bx, smem_raw);
}

// Same closed forms for L_s > 32: the band vector is staged in shared memory [L_s][blockDim].
template <typename T>
__global__ void __launch_bounds__(128) pixel_kernel_wide(PixelArgs<T> args) {
    const T* __restrict__ X = args.X;
    const T* __restrict__ BX = args.BX;
    T* __restrict__ Lam1 = args.Lam1;
    T* __restrict__ U1 = args.U1;
    T* __restrict__ Lam2 = args.Lam2;
    T* __restrict__ U2 = args.U2;
    const T* __restrict__ D9a = args.D9a;
    const T* __restrict__ D9b = args.D9b;
    const T* __restrict__ M1 = args.M1;
    const T* __restrict__ F = args.F;
    const int H = args.H, W = args.W, Ls = args.Ls, d = args.d;
    const T rho = args.rho;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* a = reinterpret_cast<T*>(smem_raw);     // [Ls][blockDim]
    const int tid = threadIdx.x, nb = blockDim.x;
    const size_t n = (size_t)H * W;
    const size_t p = (size_t)blockIdx.x * nb + tid;
    if (p >= n) return;
    for (int j = 0; j < Ls; ++j) a[j * nb + tid] = X[j * n + p] - Lam2[j * n + p] + D9b[j * n + p];
    for (int c = 0; c < Ls; ++c) {
        T acc = T(0);
        for (int j = 0; j < Ls; ++j) acc += a[j * nb + tid] * __ldg(F + j * Ls + c);
        const T w2 = X[c * n + p] - Lam2[c * n + p];
        const T l2 = acc - w2;
        Lam2[c * n + p] = l2;
        U2[c * n + p] = acc + l2;
    }
    if (args.no_p1) return;
    const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
    if (sampled_pixel(args.mask, p, y, x, d)) {
        const size_t nl = (size_t)(H / d) * (W / d);
        const size_t pl = (size_t)(y / d) * (W / d) + x / d;
        for (int j = 0; j < Ls; ++j) a[j * nb + tid] = rho * (BX[j * n + p] - Lam1[j * n + p]) + D9a[j * nl + pl];
        for (int c = 0; c < Ls; ++c) {
            T acc = T(0);
            for (int j = 0; j < Ls; ++j) acc += a[j * nb + tid] * __ldg(M1 + j * Ls + c);
            const T w1 = BX[c * n + p] - Lam1[c * n + p];
            const T l1 = acc - w1;
            Lam1[c * n + p] = l1;
            U1[c * n + p] = acc + l1;
        }
    } else {
        for (int c = 0; c < Ls; ++c) {
            const T w1 = BX[c * n + p] - Lam1[c * n + p];
            Lam1[c * n + p] = T(0);
            U1[c * n + p] = w1;
        }
    }
}

// S^T Y_l E^T / rho on the full grid: out[c][y][x] = scale lo[c][y/d][x/d] on the lattice
// y = x = 0 (mod d), 0 elsewhere (the data term of the variant with S B in the X system).
template <typename T>
__global__ void __launch_bounds__(256)
upsample_kernel(const T* __restrict__ lo, T* __restrict__ out, int H, int W, int d, int Ls, T scale) {
    const size_t n = (size_t)H * W;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * Ls) return;
    const int c = (int)(idx / n);
    const size_t pix = idx - (size_t)c * n;
    const int y = (int)(pix / W), x = (int)(pix - (size_t)y * W);
    const size_t nl = (size_t)(H / d) * (W / d);
    out[idx] = (y % d == 0 && x % d == 0) ? scale * lo[(size_t)c * nl + (size_t)(y / d) * (W / d) + x / d] : T(0);
}

// out[c][p] = sum_l in[l][p] M[l][c] for every pixel p (band mixing: S^T Y_l E^T,
// lambda1/rho Y_h R^T E^T, Z = X E).  M is Lin x Lout row-major.
template <typename T>
__global__ void __launch_bounds__(128)
band_mix_kernel(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ M, size_t npix,
                int Lin, int Lout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* a = reinterpret_cast<T*>(smem_raw);     // [Lin][blockDim]
    const int tid = threadIdx.x, nb = blockDim.x;
    const size_t p = (size_t)blockIdx.x * nb + tid;
    if (p >= npix) return;
    for (int l = 0; l < Lin; ++l) a[l * nb + tid] = in[l * npix + p];
    for (int c = 0; c < Lout; ++c) {
        T acc = T(0);
        for (int l = 0; l < Lin; ++l) acc += a[l * nb + tid] * __ldg(M + (size_t)l * Lout + c);
        out[(size_t)c * npix + p] = acc;
    }
}

}  // namespace fuse
