// Register-resident 2D DFT solve of the X system (Sec. IV-A eqs. x_linear_system_main and inv):
//   X_c = IDFT( f(w) * DFT(C_c) ),  two real bands per complex transform (see k_fft.cuh),
// for images whose sides are N = 32 P with P in {1, 2, 3, 4, 5, 6, 8, 10, 12, 16}.
//
// One warp transforms one line; lane l holds the P points n = l + 32 j (j < P), so every load and
// store of a row is a coalesced 128-byte (real) or 256-byte (complex) warp access.  With
// n = l + 32 j and k = k1 + P k2 (k1 < P, k2 < 32) the forward DFT factors as
//   Z[k1 + P k2] = sum_l w_32^{l k2} [ w_N^{l k1} sum_j z[l + 32 j] w_P^{j k1} ],   w_M = exp(-2 pi i / M):
// a P-point DFT in each lane's registers (mixed radix 4, 2, 3, 5 with the index maps resolved at
// compile time), the twist w_N^{l k1}, and for every k1 a 32-point DFT across the lanes (radix-2
// decimation in frequency, partners exchanged by warp shuffles).  Lane l then holds frequency
// k1 + P rev5(l) in slot k1 (rev5 = 5-bit reversal).  Spectra stay in this slot-major order
// (position k1 * 32 + l): the column pass works on each position independently, the factor f is
// stored in the same order by the host, and the inverse applies the adjoint of every forward step
// in reverse order (decimation in time across lanes with conjugate twiddles, the conjugate twist,
// inverse P-point DFTs), which takes the permuted spectrum back to natural order; the DFT's
// F^H F = N I makes that the unnormalised inverse, and f carries 1/(H W).
//
// Passes over band pair p (three launches, like the shared-memory form):
//   rows forward: z = C_{2p} + i C_{2p+1} along x, spectra to Y in slot-major order;
//   columns: a [H][8] tile of Y in shared memory, one warp per column: forward along y,
//            times f, inverse along y;
//   rows inverse: along x, X_{2p} = Re, X_{2p+1} = Im.
// Twiddles come from the host's FP64 tables exp(-2 pi i k / N) (k1 twists, radix-2 stage factors,
// and w_P^m = table[32 m]).
#pragma once
#include "common.cuh"
#include "k_fft.cuh"

namespace fuse {

constexpr int kWfftCols = 8;                 // columns per block of the column pass (one warp each)

__host__ __device__ constexpr bool wfft_p_ok(int P) {
    return P == 1 || P == 2 || P == 3 || P == 4 || P == 5 || P == 6 || P == 8 || P == 10 || P == 12 || P == 16;
}
__host__ __device__ constexpr bool wfft_length_ok(int N) { return N > 0 && N % 32 == 0 && wfft_p_ok(N / 32); }

template <typename T> struct vec2_of;
template <> struct vec2_of<float> { using type = float2; };
template <> struct vec2_of<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ cplx<T> ldc(const cplx<T>* p) {
    const typename vec2_of<T>::type r = *reinterpret_cast<const typename vec2_of<T>::type*>(p);
    return {r.x, r.y};
}
template <typename T>
__device__ __forceinline__ void stc(cplx<T>* p, cplx<T> v) {
    typename vec2_of<T>::type r;
    r.x = v.x;
    r.y = v.y;
    *reinterpret_cast<typename vec2_of<T>::type*>(p) = r;
}
// v * w (forward) or v * conj(w) (inverse)
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> twist(cplx<T> v, cplx<T> w) {
    if constexpr (INV) return {v.x * w.x + v.y * w.y, v.y * w.x - v.x * w.y};
    else return {v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x};
}
// -i z (forward) or +i z (inverse)
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> rot(cplx<T> z) {
    if constexpr (INV) return {-z.y, z.x};
    else return {z.y, -z.x};
}

// __ldg of a complex table entry as one vector load
template <typename T>
__device__ __forceinline__ cplx<T> ldtw(const cplx<T>* __restrict__ tw, int i) {
    const typename vec2_of<T>::type r = __ldg(reinterpret_cast<const typename vec2_of<T>::type*>(tw) + i);
    return {r.x, r.y};
}

// F-point DFT in place, F in {2, 3, 4, 5}; sum_j v_j exp(-+2 pi i j k / F).
template <typename T, int F, bool INV>
__device__ __forceinline__ void wfft_bfly(cplx<T>* v) {
    if constexpr (F == 2) {
        const cplx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (F == 3) {
        const T h = T(0.86602540378443865);                    // sin(2 pi / 3)
        const cplx<T> s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        const cplx<T> m = {v[0].x - T(0.5) * s.x, v[0].y - T(0.5) * s.y};
        const cplx<T> r0 = rot<T, INV>(d);
        const cplx<T> r = {h * r0.x, h * r0.y};
        v[0] = cadd(v[0], s);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    } else if constexpr (F == 4) {
        const cplx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const cplx<T> c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        const cplx<T> r = rot<T, INV>(d);
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, r);
        v[3] = csub(b, r);
    } else {
        static_assert(F == 5, "radix 2, 3, 4 or 5");
        const T c1 = T(0.30901699437494742), c2 = T(-0.80901699437494742);   // cos(2 pi / 5), cos(4 pi / 5)
        const T s1 = T(0.95105651629515357), s2 = T(0.58778525229247313);    // sin(2 pi / 5), sin(4 pi / 5)
        const cplx<T> a = v[0];
        const cplx<T> p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
        const cplx<T> p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
        const cplx<T> A1 = {a.x + c1 * p1.x + c2 * p2.x, a.y + c1 * p1.y + c2 * p2.y};
        const cplx<T> A2 = {a.x + c2 * p1.x + c1 * p2.x, a.y + c2 * p1.y + c1 * p2.y};
        const cplx<T> B1 = {s1 * m1.x + s2 * m2.x, s1 * m1.y + s2 * m2.y};
        const cplx<T> B2 = {s2 * m1.x - s1 * m2.x, s2 * m1.y - s1 * m2.y};
        const cplx<T> r1 = rot<T, INV>(B1), r2 = rot<T, INV>(B2);
        v[0] = {a.x + p1.x + p2.x, a.y + p1.y + p2.y};
        v[1] = cadd(A1, r1);
        v[4] = csub(A1, r1);
        v[2] = cadd(A2, r2);
        v[3] = csub(A2, r2);
    }
}

// P-point DFT of v[0..P) in natural order in and out (registers; indices fixed at compile time).
// w_P^m = tw[m TS].  Composite P = F B (F = 4 or 2): with j = j2 + B j1 and k = k1 + F k2,
//   X[k1 + F k2] = sum_{j2} w_B^{j2 k2} w_P^{j2 k1} sum_{j1} x[j2 + B j1] w_F^{j1 k1}.
template <typename T, int P, int TS, bool INV>
__device__ __forceinline__ void wfft_reg(cplx<T>* v, const cplx<T>* __restrict__ tw) {
    if constexpr (P == 1) {
        return;
    } else if constexpr (P <= 5) {
        wfft_bfly<T, P, INV>(v);
    } else {
        constexpr int F = P % 4 == 0 ? 4 : 2;
        constexpr int B = P / F;
        cplx<T> t[P];
#pragma unroll
        for (int j2 = 0; j2 < B; ++j2) {
            cplx<T> u[F];
#pragma unroll
            for (int j1 = 0; j1 < F; ++j1) u[j1] = v[j2 + B * j1];
            wfft_bfly<T, F, INV>(u);
#pragma unroll
            for (int k1 = 0; k1 < F; ++k1)
                t[j2 * F + k1] = (j2 && k1) ? twist<T, INV>(u[k1], ldtw(tw, j2 * k1 * TS)) : u[k1];
        }
#pragma unroll
        for (int k1 = 0; k1 < F; ++k1) {
            cplx<T> r[B];
#pragma unroll
            for (int j2 = 0; j2 < B; ++j2) r[j2] = t[j2 * F + k1];
            wfft_reg<T, B, TS * F, INV>(r, tw);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k1 + F * k2] = r[k2];
        }
    }
}

// Radix-2 stage factors of the cross-lane transform: for the stage exchanging lanes l and l ^ h
// (h = 16, 8, 4, 2 in ws[0..3]), w_{2h}^{l mod h} on the upper lane (bit h set), 1 on the lower.
template <typename T, int P>
__device__ __forceinline__ void wfft_stage_factors(const cplx<T>* __restrict__ tw, int lane, cplx<T>* ws) {
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const int h = 16 >> st;
        ws[st] = (lane & h) ? ldtw(tw, (lane & (h - 1)) * (16 * P / h)) : cplx<T>{T(1), T(0)};
    }
}

// Forward: P-point DFTs, twist, cross-lane decimation in frequency (natural -> slot-major).
template <typename T, int P>
__device__ __forceinline__ void wfft_forward(cplx<T>* v, const cplx<T>* __restrict__ tw, const cplx<T>* ws,
                                             int lane) {
    wfft_reg<T, P, 32, false>(v, tw);
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) v[k1] = twist<T, false>(v[k1], ldtw(tw, lane * k1));
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int h = 16 >> st;
        const T sg = (lane & h) ? T(-1) : T(1);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const T ox = __shfl_xor_sync(0xffffffffu, v[k1].x, h);
            const T oy = __shfl_xor_sync(0xffffffffu, v[k1].y, h);
            const cplx<T> t = {sg * v[k1].x + ox, sg * v[k1].y + oy};     // lower: a + b, upper: a - b
            v[k1] = st < 4 ? twist<T, false>(t, ws[st]) : t;
        }
    }
}

// Inverse (unnormalised): the adjoint of wfft_forward (slot-major -> natural).
template <typename T, int P>
__device__ __forceinline__ void wfft_inverse(cplx<T>* v, const cplx<T>* __restrict__ tw, const cplx<T>* ws,
                                             int lane) {
#pragma unroll
    for (int st = 4; st >= 0; --st) {
        const int h = 16 >> st;
        const T sg = (lane & h) ? T(-1) : T(1);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const cplx<T> m = st < 4 ? twist<T, true>(v[k1], ws[st]) : v[k1];
            const T ox = __shfl_xor_sync(0xffffffffu, m.x, h);
            const T oy = __shfl_xor_sync(0xffffffffu, m.y, h);
            v[k1] = {sg * m.x + ox, sg * m.y + oy};                      // lower: a + w* b, upper: a - w* b
        }
    }
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) v[k1] = twist<T, true>(v[k1], ldtw(tw, lane * k1));
    wfft_reg<T, P, 32, true>(v, tw);
}

// Rows forward of band pair p, row y (one warp).
template <typename T, int P>
__device__ __forceinline__ void wfft_row_fwd(const FFTArgs<T>& a, int y, int p, int lane) {
    const int W = a.W;
    const size_t n = (size_t)a.H * W;
    const T* re = a.C + (size_t)(2 * p) * n + (size_t)y * W + lane;
    const bool has_im = 2 * p + 1 < a.Ls;
    const T* im = re + n;
    cplx<T> v[P];
#pragma unroll
    for (int j = 0; j < P; ++j) v[j] = {__ldg(re + 32 * j), has_im ? __ldg(im + 32 * j) : T(0)};
    cplx<T> ws[4];
    wfft_stage_factors<T, P>(a.twW, lane, ws);
    wfft_forward<T, P>(v, a.twW, ws, lane);
    cplx<T>* out = a.Y + (size_t)p * n + (size_t)y * W + lane;
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) stc(out + 32 * k1, v[k1]);
}

// Rows inverse of band pair p, row y (one warp).
template <typename T, int P>
__device__ __forceinline__ void wfft_row_inv(const FFTArgs<T>& a, int y, int p, int lane) {
    const int W = a.W;
    const size_t n = (size_t)a.H * W;
    const cplx<T>* in = a.Y + (size_t)p * n + (size_t)y * W + lane;
    cplx<T> v[P];
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) v[k1] = ldc(in + 32 * k1);
    cplx<T> ws[4];
    wfft_stage_factors<T, P>(a.twW, lane, ws);
    wfft_inverse<T, P>(v, a.twW, ws, lane);
    T* re = a.X + (size_t)(2 * p) * n + (size_t)y * W + lane;
    const bool has_im = 2 * p + 1 < a.Ls;
    T* im = re + n;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        re[32 * j] = v[j].x;
        if (has_im) im[32 * j] = v[j].y;
    }
}

// Columns of band pair p, positions q0 = bx * 8 .. + 7 (256 threads, one warp per column):
// forward along y, times f (stored by the host as fT[q][s] for position q and slot-major row
// position s), inverse along y.  Shared tile [H][9] complex (pitch 9: conflict-free columns).
template <typename T, int P>
__device__ __forceinline__ void wfft_cols(const FFTArgs<T>& a, int bx, int p, unsigned char* smem_raw) {
    constexpr int CW = kWfftCols, PITCH = kWfftCols + 1;
    // H = 32 P rows of CW columns over the block's 256 threads: P values per thread, all loaded
    // before the first shared store
    constexpr int NL = 32 * P * CW / 256;
    static_assert(NL * 256 == 32 * P * CW, "256 threads cover the tile");
    cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw);
    const int H = a.H, W = a.W;
    const size_t n = (size_t)H * W;
    const int q0 = bx * CW;
    cplx<T>* Yp = a.Y + (size_t)p * n;
    const int cc = threadIdx.x % CW, r0 = threadIdx.x / CW;
    const bool inq = q0 + cc < W;
    cplx<T> ld[NL];
#pragma unroll
    for (int i = 0; i < NL; ++i)
        ld[i] = inq ? ldc(Yp + (size_t)(r0 + i * (256 / CW)) * W + q0 + cc) : cplx<T>{T(0), T(0)};
#pragma unroll
    for (int i = 0; i < NL; ++i) tile[(r0 + i * (256 / CW)) * PITCH + cc] = ld[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    const int q = q0 + c;
    if (c < CW && q < W) {
        cplx<T> v[P];
#pragma unroll
        for (int j = 0; j < P; ++j) v[j] = tile[(lane + 32 * j) * PITCH + c];
        cplx<T> ws[4];
        wfft_stage_factors<T, P>(a.twH, lane, ws);
        wfft_forward<T, P>(v, a.twH, ws, lane);
        const T* fq = a.fT + (size_t)q * H + lane;
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const T g = __ldg(fq + 32 * k1);
            v[k1].x *= g;
            v[k1].y *= g;
        }
        wfft_inverse<T, P>(v, a.twH, ws, lane);
#pragma unroll
        for (int j = 0; j < P; ++j) tile[(lane + 32 * j) * PITCH + c] = v[j];
    }
    __syncthreads();
    if (inq) {
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const int row = r0 + i * (256 / CW);
            stc(Yp + (size_t)row * W + q0 + cc, tile[row * PITCH + cc]);
        }
    }
}

// Occupancy of the FP32 passes: three 256-thread blocks per SM for the column pass (at most 80
// registers a thread) where its body fits in them (P <= 12), four for the row passes (64); FP64
// and larger P: the compiler's allocation.  The batched kernels take the P <= 12 bounds for every
// block (a 512 side then spills a few registers in the column pass).
template <typename T, int P>
constexpr int wfft_cols_min_blocks() { return sizeof(T) == 4 && P <= 12 ? 3 : 1; }
template <typename T, int PASS>
constexpr int fft_batch_min_blocks() { return sizeof(T) != 4 ? 1 : PASS == 1 ? 3 : 4; }

template <typename T>
__host__ __device__ constexpr size_t wfft_cols_smem(int H) {
    return (size_t)H * (kWfftCols + 1) * sizeof(cplx<T>);
}

// Single-problem kernels: rows 8 per block (one per warp), grid (ceil(H / 8), pairs); columns
// grid (ceil(W / 8), pairs).
template <typename T, int P>
__global__ void __launch_bounds__(256) wfft_rows_fwd_kernel(FFTArgs<T> a) {
    const int y = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (y < a.H) wfft_row_fwd<T, P>(a, y, blockIdx.y, threadIdx.x & 31);
}
template <typename T, int P>
__global__ void __launch_bounds__(256, (wfft_cols_min_blocks<T, P>())) wfft_cols_kernel(FFTArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    wfft_cols<T, P>(a, blockIdx.x, blockIdx.y, smem_raw);
}
template <typename T, int P>
__global__ void __launch_bounds__(256) wfft_rows_inv_kernel(FFTArgs<T> a) {
    const int y = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (y < a.H) wfft_row_inv<T, P>(a, y, blockIdx.y, threadIdx.x & 31);
}

// Batched form: one launch per pass over the segment table.  Each problem keeps the form its
// context selected (FFTArgs::fT set: register-resident, blocks of 8 rows or 8 columns; NULL:
// the shared-memory Stockham passes with the problem's rpb / CW shape), so a batch computes
// exactly what the single solves compute.  Register-form blocks dispatch on the problem's P
// (rows: W / 32, columns: H / 32).
#define FUSE_WFFT_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(8) X(10) X(12) X(16)

template <typename T, int PASS>
__global__ void __launch_bounds__(256, (fft_batch_min_blocks<T, PASS>()))
fft_batch_kernel(const FFTArgs<T>* __restrict__ args, const Segment* __restrict__ seg, int nseg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int prob, bx, by, bz;
    segment_of_block(seg, nseg, blockIdx.x, &prob, &bx, &by, &bz);
    const FFTArgs<T>& a = args[prob];        // read in place (a copy would live in local memory)
    if (a.fT == nullptr) {
        if constexpr (PASS == 0) fft_rows_fwd_body<T>(a, bx, by, smem_raw);
        else if constexpr (PASS == 1) fft_cols_body<T>(a, bx, by, smem_raw);
        else fft_rows_inv_body<T>(a, bx, by, smem_raw);
        return;
    }
    const int P = (PASS == 1 ? a.H : a.W) / 32;
    const int y = bx * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    switch (P) {
#define FUSE_WFFT_CASE(PV)                                                                   \
        case PV:                                                                             \
            if constexpr (PASS == 0) { if (y < a.H) wfft_row_fwd<T, PV>(a, y, by, lane); }   \
            else if constexpr (PASS == 1) wfft_cols<T, PV>(a, bx, by, smem_raw);             \
            else { if (y < a.H) wfft_row_inv<T, PV>(a, y, by, lane); }                       \
            break;
        FUSE_WFFT_CASES(FUSE_WFFT_CASE)
#undef FUSE_WFFT_CASE
        default: break;
    }
}

}  // namespace fuse
