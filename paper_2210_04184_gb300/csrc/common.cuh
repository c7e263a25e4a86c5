// Shared device helpers of the NLPR fusion kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace fuse {

// Circular index for a value within one period of [0, n): a in [-n, 2n).
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
// Circular index for any a.
__device__ __forceinline__ int wrapn(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
// Circular index for any a, without a division when a lies in [-n, 2n).
__device__ __forceinline__ int wrapc(int a, int n) { return (a >= -n && a < 2 * n) ? wrap1(a, n) : wrapn(a, n); }

template <typename T> struct cplx { T x, y; };

template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }

// 16-byte vector of T (4 floats or 2 doubles) for 128-bit global accesses.
template <typename T, int N> struct alignas(sizeof(T) * N) vecT { T v[N]; };

// Weight storage type -> arithmetic type.
__device__ __forceinline__ float wload(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float wconv(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float wconv(float v) { return v; }
__device__ __forceinline__ double wconv(double v) { return v; }
__device__ __forceinline__ float wload(const float* p) { return __ldg(p); }
__device__ __forceinline__ double wload(const double* p) { return __ldg(p); }

__device__ __forceinline__ void wstore(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void wstore(float* p, float v) { *p = v; }
__device__ __forceinline__ void wstore(double* p, double v) { *p = v; }

__device__ __forceinline__ float texp(float x) { return expf(x); }
__device__ __forceinline__ double texp(double x) { return exp(x); }

__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }

// The symmetric clamp clamp(u, -m, m) of the soft threshold, for a bound m >= 0 prepared once
// per weight and applied to many entries.  FP32: fmaxf then fminf.  FP64: GB300 runs FP64
// arithmetic, minimum and maximum included, at a small fraction of its FP32 rate, so the clamp
// is taken on the IEEE-754 bit patterns with integer operations instead: for non-negative
// doubles the order of the values is the order of their bit patterns read as unsigned integers,
// so |u| <= m exactly when the magnitude bits of u are at most those of m, and then the result
// is u, else m with the sign of u.  Same value as fmin(fmax(u, -m), m) for every u that is not
// NaN and every m >= 0 (the bound's sign bit is cleared, so m = -0 acts as +0).
template <typename T> struct SymBound;
template <> struct SymBound<float> {
    float m;
    __device__ __forceinline__ static SymBound of(float b) { return {b}; }
    __device__ __forceinline__ float clamp(float u) const { return fminf(fmaxf(u, -m), m); }
};
template <> struct SymBound<double> {
    unsigned long long mb;                        // magnitude bits of the bound
    __device__ __forceinline__ static SymBound of(double b) {
        return {(unsigned long long)__double_as_longlong(b) & 0x7fffffffffffffffull};
    }
    __device__ __forceinline__ double clamp(double u) const {
        const unsigned long long ub = (unsigned long long)__double_as_longlong(u);
        return (ub & 0x7fffffffffffffffull) <= mb
                   ? u
                   : __longlong_as_double((long long)(mb | (ub & 0x8000000000000000ull)));
    }
};

// Streaming (evict-first) 16-byte load/store of the latent state.
__device__ __forceinline__ vecT<float, 4> ld_stream(const vecT<float, 4>* p) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    return {{v.x, v.y, v.z, v.w}};
}
__device__ __forceinline__ void st_stream(vecT<float, 4>* p, const vecT<float, 4>& a) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
}
__device__ __forceinline__ vecT<double, 2> ld_stream(const vecT<double, 2>* p) {
    double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    return {{v.x, v.y}};
}
__device__ __forceinline__ void st_stream(vecT<double, 2>* p, const vecT<double, 2>& a) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(a.v[0], a.v[1]));
}

// Vectors of VEC elements (VEC * sizeof(T) = 16 or 32 bytes) moved as 16-byte parts.
template <typename T, int VEC>
__device__ __forceinline__ void vload(const T* p, T (&v)[VEC]) {
    constexpr int PER = 16 / sizeof(T);
#pragma unroll
    for (int q = 0; q < VEC / PER; ++q) {
        const vecT<T, PER> a = reinterpret_cast<const vecT<T, PER>*>(p)[q];
#pragma unroll
        for (int j = 0; j < PER; ++j) v[q * PER + j] = a.v[j];
    }
}
template <typename T, int VEC>
__device__ __forceinline__ void vstore(T* p, const T (&v)[VEC]) {
    constexpr int PER = 16 / sizeof(T);
#pragma unroll
    for (int q = 0; q < VEC / PER; ++q) {
        vecT<T, PER> a;
#pragma unroll
        for (int j = 0; j < PER; ++j) a.v[j] = v[q * PER + j];
        reinterpret_cast<vecT<T, PER>*>(p)[q] = a;
    }
}
template <typename T, int VEC>
__device__ __forceinline__ void vstore_stream(T* p, const T (&v)[VEC]) {
    constexpr int PER = 16 / sizeof(T);
#pragma unroll
    for (int q = 0; q < VEC / PER; ++q) {
        vecT<T, PER> a;
#pragma unroll
        for (int j = 0; j < PER; ++j) a.v[j] = v[q * PER + j];
        st_stream(reinterpret_cast<vecT<T, PER>*>(p) + q, a);
    }
}

// 16-bit fixed-point storage of the latent state relative to the entry's own threshold.
// |Sigma'| <= mu always (Sigma' = -clamp(v, -mu, mu)), so the code q = rint(Sigma' 32767 / mu)
// in [-32767, 32767] stands for q mu / 32767 (absolute error at most mu / 65534).  Thresholds
// below kMinMu act as kMinMu, so that the code arithmetic stays finite where mu = 0 (there the
// stored value is at most kMinMu instead of 0).  Codes are stored in two's complement and
// converted without conversion instructions: flipping the 16-bit sign bit gives q + 2^15 in
// [1, 65535], which placed under the exponent of 2^23 (byte permute) forms the float
// 2^23 + 2^15 + q; subtracting kBias yields q.  Adding kBias to a value in [-32767, 32767]
// rounds it to the nearest integer (ties to even: the float spacing there is 1) and leaves
// q + 2^15 in the low 16 bits.
struct FixedCode {
    static constexpr float kLevels = 32767.0f;
    static constexpr float kStep = 1.0f / 32767.0f;
    static constexpr float kBias = 8421376.0f;           // 2^23 + 2^15
    static constexpr float kMinMu = 1e-20f;
    // code e (0: low half, 1: high half) of the word w as a float
    static __device__ __forceinline__ float decode(uint32_t w, int e) {
        return __uint_as_float(__byte_perm(w ^ 0x80008000u, 0x4B000000u, e ? 0x7632u : 0x7610u)) - kBias;
    }
    // float bits whose low 16 bits are rint(c) + 2^15, for c in [-32767, 32767]
    static __device__ __forceinline__ uint32_t round_bits(float c) { return __float_as_uint(c + kBias); }
    // two codes from round_bits into one word (low half first), back in two's complement
    static __device__ __forceinline__ uint32_t pack(uint32_t lo, uint32_t hi) {
        return __byte_perm(lo, hi, 0x5410u) ^ 0x80008000u;
    }
    // both codes of a word, as decode(w, 0) and decode(w, 1)
    static __device__ __forceinline__ float2 decode2(uint32_t w) {
        const uint32_t o = w ^ 0x80008000u;
        const float2 b = make_float2(__uint_as_float(__byte_perm(o, 0x4B000000u, 0x7610u)),
                                     __uint_as_float(__byte_perm(o, 0x4B000000u, 0x7632u)));
        return __fadd2_rn(b, make_float2(-kBias, -kBias));
    }
    // the rounded codes of two values in [-32767, 32767], packed as pack(round_bits(.), round_bits(.))
    static __device__ __forceinline__ uint32_t pack2(float2 c) {
        const float2 r = __fadd2_rn(c, make_float2(kBias, kBias));
        return pack(__float_as_uint(r.x), __float_as_uint(r.y));
    }
};

// The pixels kept by the sampling operator S: the lattice i1 = i2 = 0 (mod d), or, when a mask
// is given (then d = 1), the pixels where the mask is nonzero (for example a random inpainting
// mask); S^T S is diagonal either way, which is all eq. Qh_update needs.
__device__ __forceinline__ bool sampled_pixel(const uint8_t* mask, size_t p, int y, int x, int d) {
    return mask ? mask[p] != 0 : ((y % d) == 0 && (x % d) == 0);
}

// Offsets of the search window W = [-S, S]^2 \ {0} handled by one latent block row tau1
// (blockIdx.z).  Full mode: tau1 in [-S, S], all tau2 (skipping (0,0)); state index =
// row-major index in W.
// Half mode (one offset of each +-tau pair, W+ = {tau1 > 0} U {tau1 = 0, tau2 > 0}): tau1 in
// [0, S]; state index = row-major index in W+.  Weight index is always the full-W index.
struct TauMap {
    int S;
    int half;
    // Block rows are ordered heavy first: the tau1 = 0 row, which has fewer offsets, comes last
    // so that the shortest blocks fill the tail of the launch.
    __device__ __forceinline__ int t1_of_block(int by) const {
        if (half) return by < S ? by + 1 : 0;
        return by < 2 * S ? (by < S ? by - S : by - S + 1) : 0;
    }
    __device__ __forceinline__ int nt2(int t1) const {
        return t1 == 0 ? (half ? S : 2 * S) : 2 * S + 1;
    }
    __device__ __forceinline__ int t2_of(int t1, int j) const {
        if (t1 != 0) return j - S;
        return half ? j + 1 : (j >= S ? j - S + 1 : j - S);
    }
    __device__ __forceinline__ int w_index(int t1, int t2) const {
        const int side = 2 * S + 1;
        const int cell = (t1 + S) * side + (t2 + S);
        return cell > (side * side) / 2 ? cell - 1 : cell;
    }
    __device__ __forceinline__ int s_index(int t1, int t2) const {
        if (!half) return w_index(t1, t2);
        return t1 == 0 ? t2 - 1 : S + (t1 - 1) * (2 * S + 1) + (t2 + S);
    }
};

// A batched launch is a 1D grid whose blocks are split into segments; segment s covers the
// blocks [start, start + gx*gy*gz) of problem `prob`, laid out x fastest, with block row z
// starting at z0.  Segments are sorted by start.
struct Segment {
    int prob, start, gx, gy, gz, z0;
};

__device__ __forceinline__ void segment_of_block(const Segment* __restrict__ seg, int nseg, int b, int* prob,
                                                 int* bx, int* by, int* bz) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&seg[mid].start) <= b) lo = mid; else hi = mid - 1;
    }
    const Segment s = seg[lo];
    const int id = b - s.start;
    *prob = s.prob;
    *bx = id % s.gx;
    *by = (id / s.gx) % s.gy;
    *bz = s.z0 + id / (s.gx * s.gy);
}

}  // namespace fuse
