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
// Every thread of the block must call it; nt = 0 marks a thread with no line to transform.
template <typename T>
__device__ cplx<T>* fft_smem(cplx<T>* a, cplx<T>* b, const FFTPlan& P, const cplx<T>* __restrict__ tw,
                             int sign, int t, int nt) {
    int Ns = 1;
    for (int s = 0; s < P.nst; ++s) {
        const int r = P.rad[s];
        if (nt > 0) {                    // threads without a line (nt = 0) only join the barriers
            switch (r) {
                case 4: fft_stage<T, 4>(a, b, P.N, Ns, sign, tw, t, nt); break;
                case 2: fft_stage<T, 2>(a, b, P.N, Ns, sign, tw, t, nt); break;
                case 3: fft_stage<T, 3>(a, b, P.N, Ns, sign, tw, t, nt); break;
                default: fft_stage<T, 5>(a, b, P.N, Ns, sign, tw, t, nt); break;
            }
        }
        __syncthreads();
        cplx<T>* tmp = a; a = b; b = tmp;
        Ns *= r;
    }
    return a;
}

template <typename T>
struct FFTArgs {
    const T* C;          // rows forward: real input [L_s][H][W]
    cplx<T>* Y;          // complex work array [ceil(L_s/2)][H][W]
    T* X;                // rows inverse: real output [L_s][H][W]
    const T* f;          // per-frequency factor [H][W], scaled by 1/(HW)
    int H, W, Ls;
    FFTPlan planW, planH;
    const cplx<T>* twW;
    const cplx<T>* twH;
    int rpb;             // rows per block (row passes)
    int CW;              // columns per block (column pass)
    const T* fT;         // register-resident form (k_wfft.cuh): f in the spectra's order, [W][H]
};

// Rows forward, block (bx, p): rows [bx rpb, bx rpb + rpb) of band pair p;
// z(y, .) = C_{2p}(y, .) + i C_{2p+1}(y, .), transformed along x.
template <typename T>
__device__ __forceinline__ void fft_rows_fwd_body(const FFTArgs<T>& a, int bx, int p, unsigned char* smem_raw) {
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int H = a.H, W = a.W, Ls = a.Ls, rpb = a.rpb;
    const int tpr = blockDim.x / rpb;
    const int rr = threadIdx.x / tpr, t = threadIdx.x - rr * tpr;
    const int y = bx * rpb + rr;
    const size_t n = (size_t)H * W;
    cplx<T>* b0 = sm + (size_t)rr * 2 * W;
    cplx<T>* b1 = b0 + W;
    const bool ok = y < H && rr < rpb;
    const T* re = a.C + (size_t)(2 * p) * n + (size_t)y * W;
    const bool has_im = 2 * p + 1 < Ls;
    const T* im = a.C + (size_t)(2 * p + 1) * n + (size_t)y * W;
    if (rr < rpb)
        for (int x = t; x < W; x += tpr) {
            cplx<T> z = {T(0), T(0)};
            if (ok) { z.x = re[x]; if (has_im) z.y = im[x]; }
            b0[x] = z;
        }
    __syncthreads();
    cplx<T>* res = fft_smem(b0, b1, a.planW, a.twW, -1, t, rr < rpb ? tpr : 0);
    if (ok)
        for (int x = t; x < W; x += tpr) a.Y[(size_t)p * n + (size_t)y * W + x] = res[x];
}

// Columns, block (bx, p): forward along y, multiply by f(u, v), inverse along y, for the CW
// columns starting at bx CW of band pair p (warp-major per column).
template <typename T>
__device__ __forceinline__ void fft_cols_body(const FFTArgs<T>& a, int bx, int p, unsigned char* smem_raw) {
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int H = a.H, W = a.W, CW = a.CW;
    const int tpc = blockDim.x / CW;
    const int cw = threadIdx.x / tpc, t = threadIdx.x - cw * tpc;
    const int x0 = bx * CW;
    const size_t n = (size_t)H * W;
    const int pitch = 2 * H + 1;
    cplx<T>* Yp = a.Y + (size_t)p * n;
    const int nld = blockDim.x - blockDim.x % CW;     // threads that take part in loads/stores
    if ((int)threadIdx.x < nld)
        for (int idx = threadIdx.x; idx < H * CW; idx += nld) {
            const int row = idx / CW, cc = idx - row * CW;
            const int x = x0 + cc;
            sm[(size_t)cc * pitch + row] = x < W ? Yp[(size_t)row * W + x] : cplx<T>{T(0), T(0)};
        }
    __syncthreads();
    const bool mine = cw < CW;
    cplx<T>* b0 = sm + (size_t)(mine ? cw : 0) * pitch;
    cplx<T>* b1 = b0 + H;
    cplx<T>* res = fft_smem(b0, b1, a.planH, a.twH, -1, t, mine ? tpc : 0);
    const int x = x0 + cw;
    if (mine && x < W) {
        for (int u = t; u < H; u += tpc) {
            const T g = a.f[(size_t)u * W + x];
            res[u].x *= g;
            res[u].y *= g;
        }
    }
    __syncthreads();
    cplx<T>* other = res == b0 ? b1 : b0;
    res = fft_smem(res, other, a.planH, a.twH, +1, t, mine ? tpc : 0);
    // the result buffer of column cc sits at the same parity for every column
    const int off = (int)(res - b0);
    if ((int)threadIdx.x < nld)
        for (int idx = threadIdx.x; idx < H * CW; idx += nld) {
            const int row = idx / CW, cc = idx - row * CW;
            const int xx = x0 + cc;
            if (xx < W) Yp[(size_t)row * W + xx] = sm[(size_t)cc * pitch + off + row];
        }
}

// Rows inverse, block (bx, p): X_{2p} = Re, X_{2p+1} = Im of the inverse transform along x
// (f carries 1/(HW)).
template <typename T>
__device__ __forceinline__ void fft_rows_inv_body(const FFTArgs<T>& a, int bx, int p, unsigned char* smem_raw) {
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
    const int H = a.H, W = a.W, Ls = a.Ls, rpb = a.rpb;
    const int tpr = blockDim.x / rpb;
    const int rr = threadIdx.x / tpr, t = threadIdx.x - rr * tpr;
    const int y = bx * rpb + rr;
    const size_t n = (size_t)H * W;
    cplx<T>* b0 = sm + (size_t)rr * 2 * W;
    cplx<T>* b1 = b0 + W;
    const bool ok = y < H && rr < rpb;
    if (rr < rpb)
        for (int x = t; x < W; x += tpr)
            b0[x] = ok ? a.Y[(size_t)p * n + (size_t)y * W + x] : cplx<T>{T(0), T(0)};
    __syncthreads();
    cplx<T>* res = fft_smem(b0, b1, a.planW, a.twW, +1, t, rr < rpb ? tpr : 0);
    if (!ok) return;
    T* re = a.X + (size_t)(2 * p) * n + (size_t)y * W;
    const bool has_im = 2 * p + 1 < Ls;
    T* im = a.X + (size_t)(2 * p + 1) * n + (size_t)y * W;
    for (int x = t; x < W; x += tpr) {
        re[x] = res[x].x;
        if (has_im) im[x] = res[x].y;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) fft_rows_fwd_kernel(FFTArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_rows_fwd_body<T>(a, blockIdx.x, blockIdx.y, smem_raw);
}
template <typename T>
__global__ void __launch_bounds__(256) fft_cols_kernel(FFTArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_cols_body<T>(a, blockIdx.x, blockIdx.y, smem_raw);
}
template <typename T>
__global__ void __launch_bounds__(256) fft_rows_inv_kernel(FFTArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fft_rows_inv_body<T>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// Column pass of the variant that keeps S B in the X system (not the paper's splitting):
//   (I + sum D^T D + beta d^2 B^T S^T S B) X_c = C_c,   beta = eps / (rho d^2),  E E^T = eps I.
// S^T S keeps the lattice i1 = i2 = 0 (mod d), so in the DFT basis frequency (u, v) couples with
// its d^2 aliases (u + a H/d, v + b W/d): per alias class the system is diag(g) + beta u u^H with
// u = conj(b^) and g = 1 + |P| sum_tau |d^_{tau 0}|^2.  Sherman-Morrison solves it in closed form:
//   s = sum_k p_k r_k,   x_j = q_j r_j - conj(p_j) kappa s,
// with p = b^/g, q = 1/(g H W) and kappa = beta / ((1 + beta sum_k |b^_k|^2/g_k) H W) per class,
// all precomputed on the host in FP64 (the 1/(HW) of the inverse DFT folded into q and kappa).
// The solve is C-linear, so the two real bands of a complex transform still ride together.
//
// Block (bx, p): the m base columns x0 = bx m .. bx m + m - 1 (< W/d) and, for each, its d alias
// columns x0 + j + b W/d: column cc = b m + j of the block.  Forward FFT along y of every column,
// the class solves (one thread per class (u0, j), u0 < H/d), inverse FFT along y.
template <typename T>
struct FFTAliasArgs {
    cplx<T>* Y;              // complex work array [ceil(L_s/2)][H][W], transformed along x already
    int H, W, d, m;
    FFTPlan planH;
    const cplx<T>* twH;
    const T* q;              // [H][W]
    const cplx<T>* pf;       // [H][W]
    const T* kap;            // [H/d][W/d]
};

template <typename T>
__global__ void __launch_bounds__(256) fft_cols_alias_kernel(FFTAliasArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);      // [CW][2H + 1]
    const int H = a.H, W = a.W, d = a.d, m = a.m;
    const int CW = m * d, h = H / d, w = W / d;
    const int tpc = blockDim.x / CW;
    const int cw = threadIdx.x / tpc, t = threadIdx.x - cw * tpc;
    const int x0 = blockIdx.x * m;
    const size_t n = (size_t)H * W;
    const int pitch = 2 * H + 1;
    cplx<T>* Yp = a.Y + (size_t)blockIdx.y * n;
    const int nld = blockDim.x - blockDim.x % CW;
    if ((int)threadIdx.x < nld)
        for (int idx = threadIdx.x; idx < H * CW; idx += nld) {
            const int row = idx / CW, cc = idx - row * CW;
            const int b = cc / m, j = cc - b * m;
            sm[(size_t)cc * pitch + row] =
                x0 + j < w ? Yp[(size_t)row * W + x0 + j + b * w] : cplx<T>{T(0), T(0)};
        }
    __syncthreads();
    const bool mine = cw < CW;
    cplx<T>* b0 = sm + (size_t)(mine ? cw : 0) * pitch;
    cplx<T>* b1 = b0 + H;
    cplx<T>* res = fft_smem(b0, b1, a.planH, a.twH, -1, t, mine ? tpc : 0);
    const int off = (int)(res - b0);      // the spectrum of every column sits at this offset
    for (int cls = threadIdx.x; cls < h * m; cls += blockDim.x) {
        const int u0 = cls / m, j = cls - u0 * m;
        if (x0 + j >= w) continue;
        cplx<T> s = {T(0), T(0)};
        for (int aa = 0; aa < d; ++aa)
#pragma unroll 4
            for (int bb = 0; bb < d; ++bb) {
                const int u = u0 + aa * h, x = x0 + j + bb * w;
                s = cadd(s, cmul(a.pf[(size_t)u * W + x], sm[(size_t)(bb * m + j) * pitch + off + u]));
            }
        const T kp = a.kap[(size_t)u0 * w + x0 + j];
        s.x *= kp;
        s.y *= kp;
        for (int aa = 0; aa < d; ++aa)
#pragma unroll 4
            for (int bb = 0; bb < d; ++bb) {
                const int u = u0 + aa * h, x = x0 + j + bb * w;
                const cplx<T> pv = a.pf[(size_t)u * W + x];
                const T qv = a.q[(size_t)u * W + x];
                const cplx<T> corr = cmul(cplx<T>{pv.x, -pv.y}, s);
                cplx<T>& r = sm[(size_t)(bb * m + j) * pitch + off + u];
                r = cplx<T>{qv * r.x - corr.x, qv * r.y - corr.y};
            }
    }
    __syncthreads();
    cplx<T>* other = res == b0 ? b1 : b0;
    res = fft_smem(res, other, a.planH, a.twH, +1, t, mine ? tpc : 0);
    const int off2 = (int)(res - b0);
    if ((int)threadIdx.x < nld)
        for (int idx = threadIdx.x; idx < H * CW; idx += nld) {
            const int row = idx / CW, cc = idx - row * CW;
            const int b = cc / m, j = cc - b * m;
            if (x0 + j < w) Yp[(size_t)row * W + x0 + j + b * w] = sm[(size_t)cc * pitch + off2 + row];
        }
}

}  // namespace fuse
