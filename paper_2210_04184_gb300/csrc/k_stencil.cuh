// Circular 2D blur stencils (Sec. I-A): out(i) = sum_{u,v} taps(u,v) in(i + (u,v)), with
// taps = b for B^T (correlation) and taps(u,v) = b(-u,-v) for B (convolution).
//
// MODE 0: out = stencil(in)                                        -> B X
// MODE 1: out = stencil(U1) + U2 + R,  R(j) = sum_{tau1} [A_{tau1}(j) - V_{tau1}(j + (tau1,0))]
//         (half-window mode: tau1 >= 0 only and R doubled, see k_latent.cuh)
//         the right-hand side C = B^T(P1 + Lambda1) + P2 + Lambda2 + sum D^T(Q + Sigma)
//         (Sec. IV-A, after eq. x_linear_system_main), with R from the latent pass planes.
// Tiles of 32 x 32 pixels of one band (the separable B X kernel: of several bands per block); the
// halo is loaded with circular wrap.  Blur sizes are odd and at most 15 x 15.
#pragma once
#include "common.cuh"

namespace fuse {

constexpr int ST_TX = 32, ST_TY = 32, ST_BY = 8;

// Loads the th x tw input tile whose top-left element is (y0 - rh, x0 - rw) of the H x W plane
// `in`, with circular indices, into tile[rr * pitch + cc].  When every index of the tile lies in
// [-n, 2n) (the usual case: the tile and its halo are smaller than the image) the wrap is one
// compare and select; otherwise (tiny images) the general modulo.  The test is uniform per block.
template <typename T>
__device__ __forceinline__ void load_tile(const T* __restrict__ in, int H, int W, int y0, int x0, int rh, int rw,
                                          int th, int tw, T* tile, int pitch) {
    const bool near = y0 - rh >= -H && y0 - rh + th <= 2 * H && x0 - rw >= -W && x0 - rw + tw <= 2 * W;
    if (near) {
        for (int rr = threadIdx.y; rr < th; rr += ST_BY) {
            const T* row = in + (size_t)wrap1(y0 - rh + rr, H) * W;
            for (int cc = threadIdx.x; cc < tw; cc += ST_TX) tile[rr * pitch + cc] = row[wrap1(x0 - rw + cc, W)];
        }
    } else {
        for (int rr = threadIdx.y; rr < th; rr += ST_BY) {
            const T* row = in + (size_t)wrapn(y0 - rh + rr, H) * W;
            for (int cc = threadIdx.x; cc < tw; cc += ST_TX) tile[rr * pitch + cc] = row[wrapn(x0 - rw + cc, W)];
        }
    }
}

template <typename T>
struct StencilArgs {
    const T* in;
    T* out;
    const T* taps;
    int bw, H, W;
    const T* U2;        // MODE 1 only
    const T* planes;    // MODE 1 only
    int S, half;
};

// Writes the QY outputs of one thread (rows y_first.., column x of band c); MODE 1 adds U2 and
// the adjoint sum R of the latent planes.
template <typename T, int MODE, int QY>
__device__ __forceinline__ void stencil_store(const StencilArgs<T>& a, const T (&acc)[QY], int x, int y_first, int c) {
    const int H = a.H, W = a.W, S = a.S, half = a.half;
    const size_t n = (size_t)H * W;
    const int side = 2 * S + 1;
#pragma unroll
    for (int q = 0; q < QY; ++q) {
        const int y = y_first + q;
        if (y >= H) break;
        T val = acc[q];
        const size_t pix = (size_t)y * W + x;
        if constexpr (MODE == 1) {
            const T* pc = a.planes + (size_t)c * 2 * side * n;
            T rs = T(0);
            for (int t1 = half ? 0 : -S; t1 <= S; ++t1) {
                rs += pc[(size_t)(t1 + S) * n + pix];
                rs -= pc[(size_t)(side + t1 + S) * n + (size_t)wrap1(y + t1, H) * W + x];
            }
            val += a.U2[(size_t)c * n + pix] + (half ? T(2) * rs : rs);
        }
        a.out[(size_t)c * n + pix] = val;
    }
}

// The part of four consecutive outputs (row y, columns x..x+3, x % 4 == 0, W % 4 == 0) of band c
// that does not depend on the blur: MODE 1 adds U2 and the adjoint sum R of the latent planes,
// each read as a vector of the same four columns (the same terms in the same order as
// stencil_store); MODE 0 adds nothing.  Read before the blur's tile, so these loads and the
// tile's are in flight together.
template <typename T, int MODE>
__device__ __forceinline__ void stencil_pre4(const StencilArgs<T>& a, int x, int y, int c, T (&pre)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) pre[q] = T(0);
    if constexpr (MODE == 1) {
        const int H = a.H, W = a.W, S = a.S, half = a.half;
        const size_t n = (size_t)H * W;
        const int side = 2 * S + 1;
        const size_t pix = (size_t)y * W + x;
        const T* pc = a.planes + (size_t)c * 2 * side * n;
        T rs[4] = {T(0), T(0), T(0), T(0)};
        for (int t1 = half ? 0 : -S; t1 <= S; ++t1) {
            T pa[4], pv[4];
            vload<T, 4>(pc + (size_t)(t1 + S) * n + pix, pa);
            vload<T, 4>(pc + (size_t)(side + t1 + S) * n + (size_t)wrap1(y + t1, H) * W + x, pv);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                rs[q] += pa[q];
                rs[q] -= pv[q];
            }
        }
        T u2[4];
        vload<T, 4>(a.U2 + (size_t)c * n + pix, u2);
#pragma unroll
        for (int q = 0; q < 4; ++q) pre[q] = u2[q] + (half ? T(2) * rs[q] : rs[q]);
    }
}

// Writes the four outputs acc + pre as one 16-byte vector (pre from stencil_pre4; MODE 0: acc).
template <typename T, int MODE>
__device__ __forceinline__ void stencil_store4(const StencilArgs<T>& a, const T (&acc)[4], const T (&pre)[4], int x,
                                               int y, int c) {
    const size_t pix = (size_t)y * a.W + x;
    T val[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) val[q] = MODE == 1 ? acc[q] + pre[q] : acc[q];
    vstore<T, 4>(a.out + (size_t)c * a.H * a.W + pix, val);
}

// Each thread computes QY = 4 vertically adjacent outputs; for every tap column v it holds the
// BH + QY - 1 tile values of its column in registers, so each shared-memory read feeds up to
// QY multiply-adds.  BH is a compile-time odd size (1..15); bw is a runtime odd size.
// Block (bx, by, c): the 32 x 32 tile at columns 32 bx, rows 32 by of band c.
template <typename T, int MODE, int BH>
__device__ __forceinline__ void stencil_body(const StencilArgs<T>& a, int bx, int by, int c,
                                             unsigned char* smem_raw) {
    constexpr int QY = ST_TY / ST_BY;                 // 4 outputs per thread
    constexpr int NR = BH + QY - 1;
    const int bw = a.bw, H = a.H, W = a.W;
    const int th = ST_TY + BH - 1, tw = ST_TX + bw - 1;
    T* tile = reinterpret_cast<T*>(smem_raw);         // [th][tw]
    T* tp = tile + (size_t)th * tw;                   // [BH][bw]
    constexpr int rh = BH / 2;
    const int rw = bw / 2;
    const int x0 = bx * ST_TX, y0 = by * ST_TY;
    const size_t n = (size_t)H * W;
    const T* __restrict__ inc = a.in + (size_t)c * n;
    const int tid = threadIdx.y * ST_TX + threadIdx.x;
    const int nthr = ST_TX * ST_BY;
    load_tile<T>(inc, H, W, y0, x0, rh, rw, th, tw, tile, tw);
    for (int idx = tid; idx < BH * bw; idx += nthr) tp[idx] = a.taps[idx];
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    const int ly0 = threadIdx.y * QY;                 // first of this thread's QY rows
    T acc[QY];
#pragma unroll
    for (int q = 0; q < QY; ++q) acc[q] = T(0);
    for (int v = 0; v < bw; ++v) {
        T col[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) col[r] = tile[(size_t)(ly0 + r) * tw + threadIdx.x + v];
#pragma unroll
        for (int u = 0; u < BH; ++u) {
            const T t = tp[u * bw + v];
#pragma unroll
            for (int q = 0; q < QY; ++q) acc[q] += t * col[q + u];
        }
    }
    stencil_store<T, MODE, QY>(a, acc, x, y0 + ly0, c);
}

// Square blurs (B x B, the usual case): the tap loops are unrolled at compile time and the taps
// travel in the kernel's argument space, so every multiply-add reads its tap as a constant
// operand and the tile reads use fixed offsets.
template <typename T, int B>
struct SquareTaps {
    T t[B * B];
};

// Block (bx, by, c): the 32 x 32 tile at columns 32 bx, rows 32 by of band c.
template <typename T, int MODE, int B>
__device__ __forceinline__ void stencil_sq_body(const StencilArgs<T>& a, const SquareTaps<T, B>& taps, int bx, int by,
                                                int c, unsigned char* smem_raw) {
    constexpr int QY = ST_TY / ST_BY;
    constexpr int NR = B + QY - 1;
    constexpr int TH = ST_TY + B - 1, TW = ST_TX + B - 1, R = B / 2;
    const int H = a.H, W = a.W;
    T* tile = reinterpret_cast<T*>(smem_raw);         // [TH][TW]
    const int x0 = bx * ST_TX, y0 = by * ST_TY;
    const T* __restrict__ inc = a.in + (size_t)c * H * W;
    load_tile<T>(inc, H, W, y0, x0, R, R, TH, TW, tile, TW);
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    const int ly0 = threadIdx.y * QY;
    const T* tcol = tile + ly0 * TW + threadIdx.x;
    T acc[QY];
#pragma unroll
    for (int q = 0; q < QY; ++q) acc[q] = T(0);
#pragma unroll
    for (int v = 0; v < B; ++v) {
        T col[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) col[r] = tcol[r * TW + v];
#pragma unroll
        for (int u = 0; u < B; ++u) {
#pragma unroll
            for (int q = 0; q < QY; ++q) acc[q] += taps.t[u * B + v] * col[q + u];
        }
    }
    stencil_store<T, MODE, QY>(a, acc, x, y0 + ly0, c);
}

template <typename T, int MODE, int B>
__global__ void __launch_bounds__(256) stencil_sq_kernel(StencilArgs<T> a, SquareTaps<T, B> taps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stencil_sq_body<T, MODE, B>(a, taps, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// Batched square-blur stencil: every problem of a batch shares the blur, so the taps travel in
// the argument space as in stencil_sq_kernel.
template <typename T, int MODE, int B>
__global__ void __launch_bounds__(256)
stencil_sq_batch_kernel(const StencilArgs<T>* __restrict__ args, const Segment* __restrict__ seg, int nseg,
                        SquareTaps<T, B> taps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int prob, bx, by, bz;
    segment_of_block(seg, nseg, blockIdx.x, &prob, &bx, &by, &bz);
    const StencilArgs<T> a = args[prob];
    stencil_sq_body<T, MODE, B>(a, taps, bx, by, bz, smem_raw);
}

// Separable square blurs, b(u, v) = cu(u) cv(v) (a sampled Gaussian, for example): the B x B
// stencil as a horizontal pass over the haloed tile, hs(r, x) = sum_v cv(v) tile(r, x + v) (rows
// with the vertical halo, four consecutive columns per work item), then a vertical pass,
// out(y, x) = sum_u cu(u) hs(y + u, x), again four consecutive columns per thread, so that the
// rows of hs, the latent planes, U2 and the output move as 16-byte vectors: B (2 + (B - 1)/32)
// multiply-adds per output instead of B^2.  Shared memory per band: the tile at an odd pitch
// (TW | 1, so the four-column items of a warp hit distinct banks in the first pass), then hs at
// pitch ST_TX + 4 (rows 16-byte aligned).  Needs W % 4 == 0.
template <typename T, int B>
struct SepTaps {
    T cu[B], cv[B];
};

// Offset (elements) of hs: the tile's size rounded up to a 16-byte multiple, since the rows of hs
// are read and written as 16-byte vectors.
template <typename T, int B>
__host__ __device__ constexpr int stencil_sep_hs_offset() {
    constexpr int e = (int)(16 / sizeof(T));
    return (((ST_TY + B - 1) * ((ST_TX + B - 1) | 1)) + e - 1) / e * e;
}

// Bands per block of the separable kernel: B X (MODE 0) moves little per band, so a block takes
// several bands and issues all of their tile loads before its first shared store; the right-hand
// side (MODE 1) already has its plane loads in flight and keeps one band.
template <typename T, int MODE>
__host__ __device__ constexpr int stencil_sep_bands() { return MODE == 0 ? (sizeof(T) == 4 ? 4 : 2) : 1; }

// Shared memory of one band: the haloed tile, then (16-byte aligned) the horizontal pass's rows.
template <typename T, int B>
__host__ __device__ constexpr int stencil_sep_band_elems() {
    constexpr int e = (int)(16 / sizeof(T));
    return (stencil_sep_hs_offset<T, B>() + (ST_TY + B - 1) * (ST_TX + 4) + e - 1) / e * e;
}

template <typename T, int B, int NB = 1>
constexpr size_t stencil_sep_smem() {
    return (size_t)NB * stencil_sep_band_elems<T, B>() * sizeof(T);
}

// The TH x TW tiles whose top-left element is (y0 - rh, x0 - rw), with circular indices, of bands
// c0 .. c0 + NB - 1 (those below nbands) of the planes at `in` (plane stride H W), into
// tile0 + b * stride (row pitch `pitch`); block ST_TX x ST_BY, shape fixed at compile time, so
// every load of a thread is issued before any of its shared-memory stores.  The wrap is one
// compare and select when the tile lies within one period of the plane, else the modulo.
template <typename T, int TH, int TW, int NB>
__device__ __forceinline__ void load_tiles_ct(const T* __restrict__ in, int H, int W, int c0, int nbands, int y0,
                                              int x0, int rh, int rw, T* tile0, int stride, int pitch) {
    constexpr int NR = (TH + ST_BY - 1) / ST_BY, NC = (TW + ST_TX - 1) / ST_TX;
    const bool near = y0 - rh >= -H && y0 - rh + TH <= 2 * H && x0 - rw >= -W && x0 - rw + TW <= 2 * W;
    const size_t n = (size_t)H * W;
    T v[NB][NR][NC];
    int col[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const int cc = threadIdx.x + j * ST_TX;
        col[j] = near ? wrap1(x0 - rw + cc, W) : wrapn(x0 - rw + cc, W);
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int rr = threadIdx.y + i * ST_BY;
        const size_t row = (size_t)(near ? wrap1(y0 - rh + rr, H) : wrapn(y0 - rh + rr, H)) * W;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int j = 0; j < NC; ++j)
                if (c0 + b < nbands && rr < TH && threadIdx.x + j * ST_TX < TW)
                    v[b][i][j] = in[(size_t)(c0 + b) * n + row + col[j]];
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int rr = threadIdx.y + i * ST_BY;
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                const int cc = threadIdx.x + j * ST_TX;
                if (c0 + b < nbands && rr < TH && cc < TW) tile0[b * stride + rr * pitch + cc] = v[b][i][j];
            }
        }
}

// Block (bx, by, cz): the 32 x 32 outputs at columns 32 bx, rows 32 by of the bands
// cz NB .. cz NB + NB - 1 below nbands.  Per band a horizontal pass over its haloed tile (four
// consecutive columns per work item) into its own shared rows, then the vertical pass with four
// outputs per thread.
template <typename T, int MODE, int B>
__device__ __forceinline__ void stencil_sep_body(const StencilArgs<T>& a, const SepTaps<T, B>& tp, int bx, int by,
                                                 int cz, int nbands, unsigned char* smem_raw) {
    constexpr int NB = stencil_sep_bands<T, MODE>();
    constexpr int R = B / 2;
    constexpr int TH = ST_TY + B - 1, TW = ST_TX + B - 1, TP = TW | 1, HP = ST_TX + 4;
    constexpr int CG = ST_TX / 4;                     // four-column groups per row
    constexpr int BS = stencil_sep_band_elems<T, B>();
    const int H = a.H, W = a.W;
    T* tile0 = reinterpret_cast<T*>(smem_raw);        // band b: tile [TH][TP] at b BS, then hs [TH][HP]
    const int x0 = bx * ST_TX, y0 = by * ST_TY;
    const int c0 = cz * NB;
    const int tid = threadIdx.y * ST_TX + threadIdx.x;
    const int vy = tid / CG, vx = (tid - vy * CG) * 4;
    const int x = x0 + vx, y = y0 + vy;
    const bool out = x < W && y < H;
    T pre[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
        if (out && c0 + b < nbands) stencil_pre4<T, MODE>(a, x, y, c0 + b, pre[b]);
    load_tiles_ct<T, TH, TW, NB>(a.in, H, W, c0, nbands, y0, x0, R, R, tile0, BS, TP);
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (c0 + b >= nbands) break;
        const T* tile = tile0 + b * BS;
        T* hs = tile0 + b * BS + stencil_sep_hs_offset<T, B>();    // 16-byte aligned
        for (int it = tid; it < TH * CG; it += ST_TX * ST_BY) {
            const int r = it / CG, xx = (it - r * CG) * 4;
            T w[4 + B - 1];
#pragma unroll
            for (int k = 0; k < 4 + B - 1; ++k) w[k] = tile[r * TP + xx + k];
            T o[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                o[q] = T(0);
#pragma unroll
                for (int v = 0; v < B; ++v) o[q] += tp.cv[v] * w[q + v];
            }
            vstore<T, 4>(hs + r * HP + xx, o);
        }
    }
    __syncthreads();
    if (!out) return;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (c0 + b >= nbands) break;
        const T* hs = tile0 + b * BS + stencil_sep_hs_offset<T, B>();
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int u = 0; u < B; ++u) {
            T h[4];
            vload<T, 4>(hs + (vy + u) * HP + vx, h);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += tp.cu[u] * h[q];
        }
        stencil_store4<T, MODE>(a, acc, pre[b], x, y, c0 + b);
    }
}

template <typename T, int MODE, int B>
__global__ void __launch_bounds__(256) stencil_sep_kernel(StencilArgs<T> a, SepTaps<T, B> taps, int nbands) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stencil_sep_body<T, MODE, B>(a, taps, blockIdx.x, blockIdx.y, blockIdx.z, nbands, smem_raw);
}

template <typename T, int MODE, int B>
__global__ void __launch_bounds__(256)
stencil_sep_batch_kernel(const StencilArgs<T>* __restrict__ args, const Segment* __restrict__ seg, int nseg,
                         SepTaps<T, B> taps, int nbands) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int prob, bx, by, bz;
    segment_of_block(seg, nseg, blockIdx.x, &prob, &bx, &by, &bz);
    const StencilArgs<T> a = args[prob];
    stencil_sep_body<T, MODE, B>(a, taps, bx, by, bz, nbands, smem_raw);
}

// C = G + U2 + R without a blur: the right-hand side of the variant that keeps S B in the X
// system, where the data term G = B^T S^T Y_l E^T / rho is fixed for the whole solve and
// precomputed once (in = G).  Same tiles and epilogue as the stencils.
template <typename T>
__global__ void __launch_bounds__(256) rhs_sum_kernel(StencilArgs<T> a) {
    constexpr int QY = ST_TY / ST_BY;
    const int x = blockIdx.x * ST_TX + threadIdx.x;
    if (x >= a.W) return;
    const int y0 = blockIdx.y * ST_TY + threadIdx.y * QY;
    const int c = blockIdx.z;
    const size_t n = (size_t)a.H * a.W;
    T acc[QY];
#pragma unroll
    for (int q = 0; q < QY; ++q) {
        const int y = y0 + q;
        acc[q] = y < a.H ? a.in[(size_t)c * n + (size_t)y * a.W + x] : T(0);
    }
    stencil_store<T, 1, QY>(a, acc, x, y0, c);
}

template <typename T, int MODE, int BH>
__global__ void __launch_bounds__(256) stencil_kernel(StencilArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stencil_body<T, MODE, BH>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

template <typename T, int MODE, int BH>
__global__ void __launch_bounds__(256)
stencil_batch_kernel(const StencilArgs<T>* __restrict__ args, const Segment* __restrict__ seg, int nseg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int prob, bx, by, bz;
    segment_of_block(seg, nseg, blockIdx.x, &prob, &bx, &by, &bz);
    const StencilArgs<T> a = args[prob];
    stencil_body<T, MODE, BH>(a, bx, by, bz, smem_raw);
}

}  // namespace fuse
