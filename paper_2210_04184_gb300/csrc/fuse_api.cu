// C-ABI of the NLPR multiband-fusion solver: context, host FP64 set-up, launch sequence.
// The contract of every entry point is in include/fuse.h.
#include "fuse.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "k_fft.cuh"
#include "k_latent.cuh"
#include "k_objective.cuh"
#include "k_pixel.cuh"
#include "k_stencil.cuh"
#include "k_weights.cuh"

using namespace fuse;

namespace {

constexpr int kMaxSmem = 200 * 1024;

struct Event2 { cudaEvent_t a, b; };

}  // namespace

struct fuse_ctx {
    // problem
    int H = 0, W = 0, Ll = 0, Lh = 0, Ls = 0, Lg = 0, K = 0, S = 0, d = 1, bh = 1, bw = 1;
    int nW = 0, nP = 0, npair = 0;
    size_t n = 0, nl = 0;
    double lam1 = 0, lam2 = 0, rho = 0, h = 0;
    fuse_dtype dtype = FUSE_F32, wdtype = FUSE_F32;
    size_t esz = 4, wsz = 4;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    // launch shapes
    int vec = 4, lat_Ty = 1, lat_threads = 0;
    size_t lat_smem = 0;
    int w_Ty = 1;
    size_t w_smem = 0;
    int fr_tpr = 32, fr_rpb = 1, fc_cw = 8, fc_tpc = 32;
    size_t fr_smem = 0, fc_smem = 0, st_smem = 0, px_smem = 0;
    int px_threads = 128;
    FFTPlan planH{}, planW{};
    // device memory
    void *X = nullptr, *BX = nullptr, *C = nullptr, *Y = nullptr;
    void *Lam1 = nullptr, *U1 = nullptr, *Lam2 = nullptr, *U2 = nullptr;
    void *Sig = nullptr, *planes = nullptr, *omega = nullptr, *D9a = nullptr, *D9b = nullptr;
    void *tapsT = nullptr, *tapsB = nullptr, *fpf = nullptr, *M1 = nullptr, *F = nullptr;
    void *Et = nullptr, *Mh = nullptr, *Emix = nullptr, *twH = nullptr, *twW = nullptr;
    double *objE = nullptr, *objER = nullptr, *partial = nullptr;
    size_t npartial = 0;
    void *sYl = nullptr, *sYh = nullptr, *sG = nullptr, *sX = nullptr, *sZ = nullptr;
    std::vector<void*> allocs;
    size_t sig_bytes = 0, plane_bytes = 0;
    // state flags
    bool have_weights = false, have_state = false, have_x = false;
    // errors
    fuse_status sticky = FUSE_OK;
    std::string err;
    // profiling / graphs
    bool profile = false;
    bool use_graph = true;
    std::vector<Event2> ev;
    size_t ev_used = 0;
    double latent_ms = 0.0;
    long long launches_all = 0, launches_latent = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int fault_alloc = -1, alloc_count = 0;
    // latent pass variant: 0 = register-staged loads, 1 = bulk-copy (TMA) ring
    int lat_impl = 1, lat_target = 256, lat_stages = 6;
    int lt_Ty = 1, lt_ncons = 0;
    size_t lt_smem = 0;
    int* d_err = nullptr;
    unsigned wait_limit = 1u << 22;
    // half-window latent state (one offset of each +-tau pair); 0 = full window
    int half = 1;
};

namespace {

fuse_status fail(fuse_ctx* c, fuse_status s, const std::string& msg) {
    if (c) {
        if (c->sticky == FUSE_OK) c->sticky = s;
        c->err = msg;
    }
    return s;
}

fuse_status fail_cuda(fuse_ctx* c, const char* what, cudaError_t e) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return fail(c, e == cudaErrorMemoryAllocation ? FUSE_ENOMEM : FUSE_ECUDA, buf);
}

#define CK(ctx, expr)                                              \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) return fail_cuda((ctx), #expr, e_); \
    } while (0)

#define CKL(ctx, name)                                             \
    do {                                                           \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return fail_cuda((ctx), name, e_);  \
    } while (0)

fuse_status dalloc(fuse_ctx* c, void** p, size_t bytes) {
    if (c->fault_alloc >= 0 && c->alloc_count++ == c->fault_alloc)
        return fail(c, FUSE_ENOMEM, "injected allocation failure (FUSE_FAULT_ALLOC)");
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail_cuda(c, "cudaMalloc", e);
    }
    c->allocs.push_back(*p);
    return FUSE_OK;
}

bool plan_fft(int N, FFTPlan* P) {
    P->N = N;
    P->nst = 0;
    int m = N;
    while (m % 4 == 0 && P->nst < 20) { P->rad[P->nst++] = 4; m /= 4; }
    while (m % 2 == 0 && P->nst < 20) { P->rad[P->nst++] = 2; m /= 2; }
    while (m % 3 == 0 && P->nst < 20) { P->rad[P->nst++] = 3; m /= 3; }
    while (m % 5 == 0 && P->nst < 20) { P->rad[P->nst++] = 5; m /= 5; }
    return m == 1;
}

// In-place inverse of an n x n row-major matrix (Gauss-Jordan, partial pivoting, FP64).
bool invert(std::vector<double>& A, int n) {
    std::vector<double> I(n * (size_t)n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
        if (A[(size_t)piv * n + col] == 0.0) return false;
        if (piv != col)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)piv * n + k], A[(size_t)col * n + k]);
                std::swap(I[(size_t)piv * n + k], I[(size_t)col * n + k]);
            }
        const double inv = 1.0 / A[(size_t)col * n + col];
        for (int k = 0; k < n; ++k) { A[(size_t)col * n + k] *= inv; I[(size_t)col * n + k] *= inv; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = A[(size_t)r * n + col];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)col * n + k];
                I[(size_t)r * n + k] -= f * I[(size_t)col * n + k];
            }
        }
    }
    A.swap(I);
    return true;
}

struct Shapes {
    int vec, lat_Ty, lat_threads, w_Ty, fr_tpr, fr_rpb, fc_cw, fc_tpc, px_threads;
    size_t lat_smem, w_smem, fr_smem, fc_smem, st_smem, px_smem, mix_smem_max;
};

fuse_status check_geometry(fuse_ctx* c, const fuse_geometry* g, int K, int S, int ratio, fuse_dtype dtype,
                           fuse_dtype wdtype, int bh, int bw, Shapes* sh, FFTPlan* pH, FFTPlan* pW) {
    if (!g) return fail(c, FUSE_EINVAL, "geometry is NULL");
    if (g->H < 1 || g->W < 1 || g->L_l < 1 || g->L_h < 1 || g->L_s < 1 || g->L_guide < 1)
        return fail(c, FUSE_EINVAL, "sizes must be positive");
    if (ratio < 1 || g->H % ratio || g->W % ratio) return fail(c, FUSE_EINVAL, "H and W must be divisible by ratio");
    if (K < 0 || K > 3) return fail(c, FUSE_EUNSUPPORTED, "K must be in [0, 3]");
    if (S < 1) return fail(c, FUSE_EINVAL, "S must be >= 1");
    if (2 * (K + S) + 1 > g->H || 2 * (K + S) + 1 > g->W) return fail(c, FUSE_EINVAL, "2(K+S)+1 exceeds the image");
    if (bh < 1 || bw < 1 || !(bh & 1) || !(bw & 1) || bh > g->H || bw > g->W)
        return fail(c, FUSE_EINVAL, "blur size must be odd and fit the image");
    if (bh > 15 || bw > 15) return fail(c, FUSE_EUNSUPPORTED, "blur larger than 15 x 15");
    if (dtype != FUSE_F32 && dtype != FUSE_F64) return fail(c, FUSE_EINVAL, "dtype must be F32 or F64");
    if (dtype == FUSE_F32 && wdtype != FUSE_F32 && wdtype != FUSE_BF16)
        return fail(c, FUSE_EUNSUPPORTED, "F32 context needs BF16 or F32 weights");
    if (dtype == FUSE_F64 && wdtype != FUSE_F64) return fail(c, FUSE_EUNSUPPORTED, "F64 context needs F64 weights");
    if (!plan_fft(g->H, pH) || !plan_fft(g->W, pW))
        return fail(c, FUSE_EUNSUPPORTED, "H and W must factor into 2, 3 and 5");
    const size_t esz = dtype == FUSE_F64 ? 8 : 4;
    const size_t csz = 2 * esz;
    sh->vec = (int)(16 / esz);
    if (g->W % sh->vec) return fail(c, FUSE_EUNSUPPORTED, "W must be a multiple of 4 (F32) or 2 (F64)");
    const int tpr = g->W / sh->vec;
    if (tpr > 256) return fail(c, FUSE_EUNSUPPORTED, "W too large for the latent kernel");
    sh->lat_Ty = tpr >= 128 ? 1 : 128 / tpr;
    if (sh->lat_Ty > g->H) sh->lat_Ty = g->H;
    sh->lat_threads = tpr * sh->lat_Ty;
    sh->lat_smem = (size_t)(2 * S + 1) * sh->lat_Ty * g->W * esz;
    if (sh->lat_smem > kMaxSmem) return fail(c, FUSE_EUNSUPPORTED, "latent tile exceeds shared memory");
    // weights
    int wt = (int)(96 * 1024 / (2 * (size_t)g->W * esz)) - 2 * K;
    sh->w_Ty = wt < 1 ? 1 : (wt > 32 ? 32 : wt);
    sh->w_smem = 2 * (size_t)(sh->w_Ty + 2 * K) * g->W * esz;
    if (sh->w_smem > kMaxSmem) return fail(c, FUSE_EUNSUPPORTED, "weights tile exceeds shared memory");
    // fft rows
    int t = g->W / 4;
    t = t < 32 ? 32 : (t > 256 ? 256 : t);
    sh->fr_tpr = t;
    sh->fr_rpb = 256 / t;
    while (sh->fr_rpb > 1 && 2 * (size_t)sh->fr_rpb * g->W * csz > 64 * 1024) sh->fr_rpb--;
    sh->fr_smem = 2 * (size_t)sh->fr_rpb * g->W * csz;
    if (sh->fr_smem > kMaxSmem) return fail(c, FUSE_EUNSUPPORTED, "W too large for the FFT");
    // fft columns
    sh->fc_cw = dtype == FUSE_F64 ? 4 : 8;
    while (sh->fc_cw > 1 && (size_t)sh->fc_cw * (2 * g->H + 1) * csz > kMaxSmem) sh->fc_cw /= 2;
    sh->fc_smem = (size_t)sh->fc_cw * (2 * g->H + 1) * csz;
    if (sh->fc_smem > kMaxSmem) return fail(c, FUSE_EUNSUPPORTED, "H too large for the FFT");
    int tc = g->H / 4;
    tc = tc < 8 ? 8 : tc;
    while (sh->fc_cw * tc > 256) tc /= 2;
    sh->fc_tpc = tc;
    // stencil
    sh->st_smem = ((size_t)(ST_TY + bh - 1) * (ST_TX + bw - 1) + (size_t)bh * bw) * esz;
    if (sh->st_smem > kMaxSmem) return fail(c, FUSE_EUNSUPPORTED, "blur too large");
    // pixel / band mixing
    sh->px_threads = 128;
    if (g->L_s <= 32) {
        sh->px_smem = 2 * (size_t)g->L_s * g->L_s * esz;
    } else {
        while (sh->px_threads > 32 && (size_t)g->L_s * sh->px_threads * esz > 96 * 1024) sh->px_threads /= 2;
        sh->px_smem = (size_t)g->L_s * sh->px_threads * esz;
    }
    int lmax = g->L_l > g->L_h ? g->L_l : g->L_h;
    if (g->L_s > lmax) lmax = g->L_s;
    sh->mix_smem_max = (size_t)lmax * 32 * esz;
    if (sh->px_smem > kMaxSmem || sh->mix_smem_max > kMaxSmem) return fail(c, FUSE_EUNSUPPORTED, "too many bands");
    return FUSE_OK;
}

size_t mix_threads(int Lin, size_t esz) {
    int t = 128;
    while (t > 32 && (size_t)Lin * t * esz > 96 * 1024) t /= 2;
    return (size_t)t;
}

struct Sizes {
    size_t img, cimg, sig, planes, omega, d9a;
};

Sizes sizes_of(const fuse_geometry* g, int K, int S, int ratio, size_t esz, size_t wsz, int half = 1) {
    Sizes z;
    const size_t n = (size_t)g->H * g->W;
    const size_t nW = (size_t)(2 * S + 1) * (2 * S + 1) - 1, nP = (size_t)(2 * K + 1) * (2 * K + 1);
    z.img = n * g->L_s * esz;
    z.cimg = n * ((g->L_s + 1) / 2) * 2 * esz;
    z.sig = (half ? nW / 2 : nW) * nP * g->L_s * n * esz;
    z.planes = (size_t)g->L_s * 2 * (2 * S + 1) * n * esz;
    z.omega = nW * n * wsz;
    z.d9a = (size_t)g->L_s * (n / ((size_t)ratio * ratio)) * esz;
    return z;
}

// Launch shape of the bulk-copy latent pass: about `target` consumer threads per block (full
// rows), `stages` ring slots; false if it does not fit in shared memory.
bool latent_tma_shape(fuse_ctx* c) {
    const int tpr = c->W / c->vec;
    int Ty = c->lat_target / tpr;
    if (Ty < 1) Ty = 1;
    if (Ty > c->H) Ty = c->H;
    while (Ty > 1 && ((tpr * Ty + 31) / 32) * 32 + 32 > 288) --Ty;
    const int ncons = ((tpr * Ty + 31) / 32) * 32;
    if (ncons + 32 > 288) return false;
    const size_t smem = (size_t)(c->lat_stages + 2 * c->S + 1) * Ty * c->W * c->esz + 2 * (size_t)c->lat_stages * 8;
    if (smem > (size_t)kMaxSmem || c->lat_stages < 1) return false;
    c->lt_Ty = Ty;
    c->lt_ncons = ncons;
    c->lt_smem = smem;
    return true;
}

// ---------------------------------------------------------------------------------------
// typed launch sequence
// ---------------------------------------------------------------------------------------

template <typename T>
struct Impl {
    static fuse_status set_attrs(fuse_ctx* c) {
        CK(c, cudaFuncSetAttribute(fft_rows_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->fr_smem));
        CK(c, cudaFuncSetAttribute(fft_rows_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->fr_smem));
        CK(c, cudaFuncSetAttribute(fft_cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->fc_smem));

        CK(c, cudaFuncSetAttribute(pixel_kernel_wide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->px_smem));
        if (stencil_attr(c) != FUSE_OK) return c->sticky;
        CK(c, cudaFuncSetAttribute(band_mix_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        return FUSE_OK;
    }

    template <typename WT>
    static fuse_status set_attrs_w(fuse_ctx* c) {
        CK(c, cudaFuncSetAttribute(weights_kernel<T, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->w_smem));
        constexpr int V = 16 / sizeof(T);
        const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        switch (c->K) {
            case 0: CK(c, cudaFuncSetAttribute(latent_kernel<T, WT, 0, V>, A, (int)c->lat_smem));
                    CK(c, cudaFuncSetAttribute(latent_tma_kernel<T, WT, 0, V>, A, kMaxSmem)); break;
            case 1: CK(c, cudaFuncSetAttribute(latent_kernel<T, WT, 1, V>, A, (int)c->lat_smem));
                    CK(c, cudaFuncSetAttribute(latent_tma_kernel<T, WT, 1, V>, A, kMaxSmem)); break;
            case 2: CK(c, cudaFuncSetAttribute(latent_kernel<T, WT, 2, V>, A, (int)c->lat_smem));
                    CK(c, cudaFuncSetAttribute(latent_tma_kernel<T, WT, 2, V>, A, kMaxSmem)); break;
            default: CK(c, cudaFuncSetAttribute(latent_kernel<T, WT, 3, V>, A, (int)c->lat_smem));
                     CK(c, cudaFuncSetAttribute(latent_tma_kernel<T, WT, 3, V>, A, kMaxSmem)); break;
        }
        return FUSE_OK;
    }

    template <int MODE, int BH>
    static void stencil_bh(fuse_ctx* c, cudaStream_t s, const void* in, void* out, const void* taps) {
        dim3 grid((unsigned)((c->W + ST_TX - 1) / ST_TX), (unsigned)((c->H + ST_TY - 1) / ST_TY), (unsigned)c->Ls);
        stencil_kernel<T, MODE, BH><<<grid, dim3(ST_TX, ST_BY), c->st_smem, s>>>(
            (const T*)in, (T*)out, (const T*)taps, c->bw, c->H, c->W, (const T*)c->U2, (const T*)c->planes, c->S,
            c->half);
    }

    // MODE 0: out = B in (taps = flipped b); MODE 1: C = B^T U1 + U2 + R (taps = b).
    template <int MODE>
    static void stencil(fuse_ctx* c, cudaStream_t s, const void* in, void* out, const void* taps) {
        switch (c->bh) {
            case 1: stencil_bh<MODE, 1>(c, s, in, out, taps); break;
            case 3: stencil_bh<MODE, 3>(c, s, in, out, taps); break;
            case 5: stencil_bh<MODE, 5>(c, s, in, out, taps); break;
            case 7: stencil_bh<MODE, 7>(c, s, in, out, taps); break;
            case 9: stencil_bh<MODE, 9>(c, s, in, out, taps); break;
            case 11: stencil_bh<MODE, 11>(c, s, in, out, taps); break;
            case 13: stencil_bh<MODE, 13>(c, s, in, out, taps); break;
            default: stencil_bh<MODE, 15>(c, s, in, out, taps); break;
        }
    }

    template <int BH>
    static fuse_status stencil_attr_bh(fuse_ctx* c) {
        CK(c, cudaFuncSetAttribute(stencil_kernel<T, 0, BH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->st_smem));
        CK(c, cudaFuncSetAttribute(stencil_kernel<T, 1, BH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->st_smem));
        return FUSE_OK;
    }

    static fuse_status stencil_attr(fuse_ctx* c) {
        switch (c->bh) {
            case 1: return stencil_attr_bh<1>(c);
            case 3: return stencil_attr_bh<3>(c);
            case 5: return stencil_attr_bh<5>(c);
            case 7: return stencil_attr_bh<7>(c);
            case 9: return stencil_attr_bh<9>(c);
            case 11: return stencil_attr_bh<11>(c);
            case 13: return stencil_attr_bh<13>(c);
            default: return stencil_attr_bh<15>(c);
        }
    }

    static fuse_status band_mix(fuse_ctx* c, cudaStream_t s, const void* in, void* out, const void* M, size_t npix,
                                int Lin, int Lout) {
        const size_t t = mix_threads(Lin, sizeof(T));
        const unsigned blocks = (unsigned)((npix + t - 1) / t);
        band_mix_kernel<T><<<blocks, (unsigned)t, Lin * t * sizeof(T), s>>>(
            (const T*)in, (T*)out, (const T*)M, npix, Lin, Lout);
        c->launches_all++;
        CKL(c, "band_mix_kernel");
        return FUSE_OK;
    }

    template <typename WT>
    static fuse_status weights(fuse_ctx* c, const void* G) {
        dim3 grid((unsigned)((c->H + c->w_Ty - 1) / c->w_Ty), (unsigned)c->nW);
        weights_kernel<T, WT><<<grid, 256, c->w_smem, c->stream>>>(
            (const T*)G, (WT*)c->omega, c->H, c->W, c->Lg, c->K, c->S, c->w_Ty, (T)(1.0 / (c->h * c->h)));
        c->launches_all++;
        CKL(c, "weights_kernel");
        return FUSE_OK;
    }

    template <typename WT, int K>
    static void launch_latent(fuse_ctx* c, cudaStream_t s) {
        constexpr int VEC = 16 / sizeof(T);
        const unsigned rowsW = (unsigned)(c->half ? c->S + 1 : 2 * c->S + 1);
        dim3 grid((unsigned)((c->H + c->lat_Ty - 1) / c->lat_Ty), (unsigned)c->Ls, rowsW);
        latent_kernel<T, WT, K, VEC><<<grid, c->lat_threads, c->lat_smem, s>>>(
            (const T*)c->X, (const WT*)c->omega, (T*)c->Sig, (T*)c->planes, c->H, c->W, c->Ls, c->S, c->lat_Ty,
            (T)(c->lam2 / c->rho), c->half);
    }

    template <typename WT, int K>
    static void launch_latent_tma(fuse_ctx* c, cudaStream_t s) {
        constexpr int VEC = 16 / sizeof(T);
        const unsigned rowsW = (unsigned)(c->half ? c->S + 1 : 2 * c->S + 1);
        dim3 grid((unsigned)((c->H + c->lt_Ty - 1) / c->lt_Ty), (unsigned)c->Ls, rowsW);
        latent_tma_kernel<T, WT, K, VEC><<<grid, c->lt_ncons + 32, c->lt_smem, s>>>(
            (const T*)c->X, (const WT*)c->omega, (T*)c->Sig, (T*)c->planes, c->H, c->W, c->Ls, c->S, c->lt_Ty,
            c->lt_ncons, c->lat_stages, (T)(c->lam2 / c->rho), c->d_err, c->wait_limit, c->half);
    }

    template <typename WT>
    static void latent(fuse_ctx* c, cudaStream_t s) {
        if (c->lat_impl == 1) {
            switch (c->K) {
                case 0: launch_latent_tma<WT, 0>(c, s); break;
                case 1: launch_latent_tma<WT, 1>(c, s); break;
                case 2: launch_latent_tma<WT, 2>(c, s); break;
                default: launch_latent_tma<WT, 3>(c, s); break;
            }
            return;
        }
        switch (c->K) {
            case 0: launch_latent<WT, 0>(c, s); break;
            case 1: launch_latent<WT, 1>(c, s); break;
            case 2: launch_latent<WT, 2>(c, s); break;
            default: launch_latent<WT, 3>(c, s); break;
        }
    }

    static void latent_any(fuse_ctx* c, cudaStream_t s);

    // One ADMM iteration (Sec. IV): C, X update, P1/P2/duals, latent pass.
    static fuse_status iterate(fuse_ctx* c, cudaStream_t s, bool timed) {
        const size_t n = c->n;
        stencil<1>(c, s, c->U1, c->C, c->tapsT);
        dim3 rgrid((unsigned)((c->H + c->fr_rpb - 1) / c->fr_rpb), (unsigned)c->npair);
        fft_rows_fwd_kernel<T><<<rgrid, c->fr_tpr * c->fr_rpb, c->fr_smem, s>>>(
            (const T*)c->C, (cplx<T>*)c->Y, c->H, c->W, c->Ls, c->planW, (const cplx<T>*)c->twW, c->fr_rpb);
        dim3 cgrid((unsigned)((c->W + c->fc_cw - 1) / c->fc_cw), (unsigned)c->npair);
        fft_cols_kernel<T><<<cgrid, c->fc_cw * c->fc_tpc, c->fc_smem, s>>>(
            (cplx<T>*)c->Y, (const T*)c->fpf, c->H, c->W, c->planH, (const cplx<T>*)c->twH, c->fc_cw);
        fft_rows_inv_kernel<T><<<rgrid, c->fr_tpr * c->fr_rpb, c->fr_smem, s>>>(
            (const cplx<T>*)c->Y, (T*)c->X, c->H, c->W, c->Ls, c->planW, (const cplx<T>*)c->twW, c->fr_rpb);
        stencil<0>(c, s, c->X, c->BX, c->tapsB);
        const unsigned pblocks = (unsigned)((n + c->px_threads - 1) / c->px_threads);
        const T rho = (T)c->rho;
#define FUSE_PIXEL_ARGS (const T*)c->X, (const T*)c->BX, (T*)c->Lam1, (T*)c->U1, (T*)c->Lam2, (T*)c->U2, \
    (const T*)c->D9a, (const T*)c->D9b, (const T*)c->M1, (const T*)c->F, c->H, c->W, c->Ls, c->d, rho
        if (c->Ls <= 4) pixel_kernel<T, 4><<<pblocks, c->px_threads, c->px_smem, s>>>(FUSE_PIXEL_ARGS);
        else if (c->Ls <= 8) pixel_kernel<T, 8><<<pblocks, c->px_threads, c->px_smem, s>>>(FUSE_PIXEL_ARGS);
        else if (c->Ls <= 16) pixel_kernel<T, 16><<<pblocks, c->px_threads, c->px_smem, s>>>(FUSE_PIXEL_ARGS);
        else if (c->Ls <= 20) pixel_kernel<T, 20><<<pblocks, c->px_threads, c->px_smem, s>>>(FUSE_PIXEL_ARGS);
        else if (c->Ls <= 32) pixel_kernel<T, 32><<<pblocks, c->px_threads, c->px_smem, s>>>(FUSE_PIXEL_ARGS);
        else pixel_kernel_wide<T><<<pblocks, c->px_threads, c->px_smem, s>>>(FUSE_PIXEL_ARGS);
#undef FUSE_PIXEL_ARGS
        if (timed) {
            if (c->ev_used == c->ev.size()) {
                Event2 e{};
                CK(c, cudaEventCreate(&e.a));
                CK(c, cudaEventCreate(&e.b));
                c->ev.push_back(e);
            }
            Event2& e = c->ev[c->ev_used++];
            CK(c, cudaEventRecord(e.a, s));
            latent_any(c, s);
            CK(c, cudaEventRecord(e.b, s));
        } else {
            latent_any(c, s);
        }
        CKL(c, "iteration kernels");
        return FUSE_OK;
    }

    static fuse_status objective(fuse_ctx* c, const void* Yl, const void* Yh, double out[4]);
};

template <typename T>
void Impl<T>::latent_any(fuse_ctx* c, cudaStream_t s) {
    if constexpr (sizeof(T) == 8) {
        latent<double>(c, s);
    } else {
        if (c->wdtype == FUSE_BF16) latent<__nv_bfloat16>(c, s);
        else latent<float>(c, s);
    }
}

template <typename T>
fuse_status Impl<T>::objective(fuse_ctx* c, const void* Yl, const void* Yh, double out[4]) {
    const size_t n = c->n;
    stencil<0>(c, c->stream, c->X, c->BX, c->tapsB);
    const unsigned nb = (unsigned)((n + 255) / 256);
    obj_data_kernel<T><<<nb, 256, 0, c->stream>>>((const T*)c->X, (const T*)c->BX, (const T*)Yl, (const T*)Yh,
                                                   c->objE, c->objER, c->H, c->W, c->d, c->Ls, c->Ll, c->Lh,
                                                   c->partial);
    double* phi_part = c->partial + (size_t)nb * 3;
    dim3 pgrid(nb, (unsigned)c->nW);
    if constexpr (sizeof(T) == 8) {
        obj_phi_kernel<T, double><<<pgrid, 256, 0, c->stream>>>((const T*)c->X, (const double*)c->omega, c->H, c->W,
                                                                c->Ls, c->K, c->S, phi_part);
    } else {
        if (c->wdtype == FUSE_BF16)
            obj_phi_kernel<T, __nv_bfloat16><<<pgrid, 256, 0, c->stream>>>(
                (const T*)c->X, (const __nv_bfloat16*)c->omega, c->H, c->W, c->Ls, c->K, c->S, phi_part);
        else
            obj_phi_kernel<T, float><<<pgrid, 256, 0, c->stream>>>((const T*)c->X, (const float*)c->omega, c->H, c->W,
                                                                   c->Ls, c->K, c->S, phi_part);
    }
    c->launches_all += 3;
    CKL(c, "objective kernels");
    const size_t np = (size_t)nb * 3 + (size_t)nb * c->nW;
    std::vector<double> h(np);
    CK(c, cudaMemcpyAsync(h.data(), c->partial, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    double s0 = 0, s1 = 0, s3 = 0, s2 = 0;
    for (unsigned b = 0; b < nb; ++b) { s0 += h[b * 3 + 0]; s1 += h[b * 3 + 1]; s3 += h[b * 3 + 2]; }
    for (size_t q = (size_t)nb * 3; q < np; ++q) s2 += h[q];
    out[0] = 0.5 * s0;
    out[1] = 0.5 * c->lam1 * s1;
    out[2] = c->lam2 * s2;
    out[3] = s3;
    for (int q = 0; q < 4; ++q)
        if (!std::isfinite(out[q])) return fail(c, FUSE_ENONFINITE, "objective term is not finite");
    return FUSE_OK;
}

fuse_status guard(fuse_ctx* c) {
    if (!c) return FUSE_EINVAL;
    if (c->sticky != FUSE_OK) return FUSE_ESTATE;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail_cuda(c, "cudaSetDevice", e);
    return FUSE_OK;
}

fuse_status zero_state(fuse_ctx* c, cudaStream_t s) {
    const size_t img = c->n * c->Ls * c->esz;
    CK(c, cudaMemsetAsync(c->Lam1, 0, img, s));
    CK(c, cudaMemsetAsync(c->U1, 0, img, s));
    CK(c, cudaMemsetAsync(c->Lam2, 0, img, s));
    CK(c, cudaMemsetAsync(c->U2, 0, img, s));
    CK(c, cudaMemsetAsync(c->X, 0, img, s));
    CK(c, cudaMemsetAsync(c->Sig, 0, c->sig_bytes, s));
    CK(c, cudaMemsetAsync(c->planes, 0, c->plane_bytes, s));
    return FUSE_OK;
}

fuse_status run_iterations(fuse_ctx* c, int iters) {
    if (iters <= 0) return FUSE_OK;
    const bool f64 = c->dtype == FUSE_F64;
    if (c->profile || !c->use_graph) {
        for (int t = 0; t < iters; ++t) {
            fuse_status st = f64 ? Impl<double>::iterate(c, c->stream, c->profile)
                                 : Impl<float>::iterate(c, c->stream, c->profile);
            if (st != FUSE_OK) return st;
            c->launches_all += 7;
            c->launches_latent += 1;
        }
        return FUSE_OK;
    }
    if (!c->gexec) {
        CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        fuse_status st = f64 ? Impl<double>::iterate(c, c->cap_stream, false) : Impl<float>::iterate(c, c->cap_stream, false);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (st != FUSE_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return fail_cuda(c, "cudaStreamEndCapture", e);
        c->graph = g;
        CK(c, cudaGraphInstantiate(&c->gexec, c->graph, 0));
    }
    for (int t = 0; t < iters; ++t) {
        CK(c, cudaGraphLaunch(c->gexec, c->stream));
        c->launches_all += 7;
        c->launches_latent += 1;
    }
    return FUSE_OK;
}

fuse_status solve_impl(fuse_ctx* c, const void* Yl, const void* Yh, int iters, int warm, void* Xo, void* Zo) {
    const bool f64 = c->dtype == FUSE_F64;
    fuse_status st;
    // S^T Y_l E^T on the sampled lattice and lambda1/rho Y_h R^T E^T (eqs. Qh_update, Qm_update)
    st = f64 ? Impl<double>::band_mix(c, c->stream, Yl, c->D9a, c->Et, c->nl, c->Ll, c->Ls)
             : Impl<float>::band_mix(c, c->stream, Yl, c->D9a, c->Et, c->nl, c->Ll, c->Ls);
    if (st != FUSE_OK) return st;
    st = f64 ? Impl<double>::band_mix(c, c->stream, Yh, c->D9b, c->Mh, c->n, c->Lh, c->Ls)
             : Impl<float>::band_mix(c, c->stream, Yh, c->D9b, c->Mh, c->n, c->Lh, c->Ls);
    if (st != FUSE_OK) return st;
    if (!warm || !c->have_state) {
        st = zero_state(c, c->stream);
        if (st != FUSE_OK) return st;
        c->have_state = true;
    }
    st = run_iterations(c, iters);
    if (st != FUSE_OK) return st;
    c->have_x = true;
    const size_t img = c->n * c->Ls * c->esz;
    if (Xo) CK(c, cudaMemcpyAsync(Xo, c->X, img, cudaMemcpyDeviceToDevice, c->stream));
    if (Zo) {
        st = f64 ? Impl<double>::band_mix(c, c->stream, c->X, Zo, c->Emix, c->n, c->Ls, c->Ll)
                 : Impl<float>::band_mix(c, c->stream, c->X, Zo, c->Emix, c->n, c->Ls, c->Ll);
        if (st != FUSE_OK) return st;
    }
    return FUSE_OK;
}

fuse_status weights_impl(fuse_ctx* c, const void* G) {
    fuse_status st;
    if (c->dtype == FUSE_F64) st = Impl<double>::weights<double>(c, G);
    else if (c->wdtype == FUSE_BF16) st = Impl<float>::weights<__nv_bfloat16>(c, G);
    else st = Impl<float>::weights<float>(c, G);
    if (st == FUSE_OK) c->have_weights = true;
    return st;
}

void release(fuse_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (auto& e : c->ev) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (void* p : c->allocs)
        if (p) cudaFree(p);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->allocs.clear();
}

template <typename T>
fuse_status upload(fuse_ctx* c, void** dst, const std::vector<double>& v) {
    std::vector<T> h(v.size());
    for (size_t i = 0; i < v.size(); ++i) h[i] = (T)v[i];
    fuse_status st = dalloc(c, dst, h.size() * sizeof(T));
    if (st != FUSE_OK) return st;
    CK(c, cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FUSE_OK;
}

fuse_status upload_any(fuse_ctx* c, void** dst, const std::vector<double>& v) {
    return c->dtype == FUSE_F64 ? upload<double>(c, dst, v) : upload<float>(c, dst, v);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------------------

extern "C" {

const char* fuse_status_string(fuse_status s) {
    switch (s) {
        case FUSE_OK: return "FUSE_OK";
        case FUSE_EINVAL: return "FUSE_EINVAL";
        case FUSE_ENOMEM: return "FUSE_ENOMEM";
        case FUSE_ECUDA: return "FUSE_ECUDA";
        case FUSE_ETIMEOUT: return "FUSE_ETIMEOUT";
        case FUSE_ENONFINITE: return "FUSE_ENONFINITE";
        case FUSE_ESTATE: return "FUSE_ESTATE";
        case FUSE_EUNSUPPORTED: return "FUSE_EUNSUPPORTED";
    }
    return "FUSE_UNKNOWN";
}

fuse_status fuse_workspace_bytes(const fuse_geometry* g, int K, int S, int ratio, fuse_dtype dtype,
                                 fuse_dtype wdtype, size_t* bytes) {
    if (!bytes) return FUSE_EINVAL;
    Shapes sh;
    FFTPlan pH, pW;
    fuse_status st = check_geometry(nullptr, g, K, S, ratio, dtype, wdtype, 1, 1, &sh, &pH, &pW);
    if (st != FUSE_OK) return st;
    const size_t esz = dtype == FUSE_F64 ? 8 : 4;
    const size_t wsz = wdtype == FUSE_BF16 ? 2 : (wdtype == FUSE_F64 ? 8 : 4);
    Sizes z = sizes_of(g, K, S, ratio, esz, wsz);
    *bytes = 7 * z.img + z.cimg + z.sig + z.planes + z.omega + z.d9a;
    return FUSE_OK;
}

fuse_status fuse_init(fuse_ctx** out, const fuse_geometry* g, const double* blur, int bh, int bw, int ratio,
                      const double* R, const double* E, int K, int S, double lambda1, double lambda2, double rho,
                      double h, fuse_dtype dtype, fuse_dtype wdtype, void* stream) {
    if (!out) return FUSE_EINVAL;
    *out = nullptr;
    if (!blur || !R) return FUSE_EINVAL;
    if (!(lambda1 > 0) || !(rho > 0) || !(h > 0) || !(lambda2 >= 0) || !std::isfinite(lambda1) ||
        !std::isfinite(lambda2) || !std::isfinite(rho) || !std::isfinite(h))
        return FUSE_EINVAL;
    Shapes sh;
    FFTPlan pH, pW;
    fuse_status st = check_geometry(nullptr, g, K, S, ratio, dtype, wdtype, bh, bw, &sh, &pH, &pW);
    if (st != FUSE_OK) return st;
    if (!E && g->L_s != g->L_l) return FUSE_EINVAL;

    fuse_ctx* c = new (std::nothrow) fuse_ctx();
    if (!c) return FUSE_ENOMEM;
    if (const char* fa = std::getenv("FUSE_FAULT_ALLOC")) c->fault_alloc = std::atoi(fa);
    c->H = g->H; c->W = g->W; c->Ll = g->L_l; c->Lh = g->L_h; c->Ls = g->L_s; c->Lg = g->L_guide;
    c->K = K; c->S = S; c->d = ratio; c->bh = bh; c->bw = bw;
    c->nW = (2 * S + 1) * (2 * S + 1) - 1;
    c->nP = (2 * K + 1) * (2 * K + 1);
    c->npair = (g->L_s + 1) / 2;
    c->n = (size_t)g->H * g->W;
    c->nl = c->n / ((size_t)ratio * ratio);
    c->lam1 = lambda1; c->lam2 = lambda2; c->rho = rho; c->h = h;
    c->dtype = dtype; c->wdtype = wdtype;
    c->esz = dtype == FUSE_F64 ? 8 : 4;
    c->wsz = wdtype == FUSE_BF16 ? 2 : (wdtype == FUSE_F64 ? 8 : 4);
    c->stream = (cudaStream_t)stream;
    c->vec = sh.vec; c->lat_Ty = sh.lat_Ty; c->lat_threads = sh.lat_threads; c->lat_smem = sh.lat_smem;
    c->w_Ty = sh.w_Ty; c->w_smem = sh.w_smem;
    c->fr_tpr = sh.fr_tpr; c->fr_rpb = sh.fr_rpb; c->fr_smem = sh.fr_smem;
    c->fc_cw = sh.fc_cw; c->fc_tpc = sh.fc_tpc; c->fc_smem = sh.fc_smem;
    c->st_smem = sh.st_smem; c->px_smem = sh.px_smem; c->px_threads = sh.px_threads;
    c->planH = pH; c->planW = pW;

    auto bail = [&](fuse_status s) { release(c); delete c; return s; };
    if (cudaGetDevice(&c->device) != cudaSuccess) { cudaGetLastError(); return bail(FUSE_ECUDA); }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return bail(FUSE_ECUDA);
    }

    // ---- host FP64 set-up ----
    const int H = c->H, W = c->W, Ls = c->Ls, Ll = c->Ll, Lh = c->Lh;
    std::vector<double> Em((size_t)Ls * Ll, 0.0);
    if (E) for (size_t i = 0; i < Em.size(); ++i) Em[i] = E[i];
    else for (int i = 0; i < Ls; ++i) Em[(size_t)i * Ll + i] = 1.0;
    std::vector<double> Rm(R, R + (size_t)Ll * Lh);
    for (double v : Em) if (!std::isfinite(v)) return bail(FUSE_EINVAL);
    for (double v : Rm) if (!std::isfinite(v)) return bail(FUSE_EINVAL);
    // taps: B^T is correlation with b, B is correlation with the flipped kernel
    std::vector<double> tT((size_t)bh * bw), tB((size_t)bh * bw);
    for (int a = 0; a < bh; ++a)
        for (int b = 0; b < bw; ++b) {
            tT[(size_t)a * bw + b] = blur[(size_t)a * bw + b];
            tB[(size_t)a * bw + b] = blur[(size_t)(bh - 1 - a) * bw + (bw - 1 - b)];
            if (!std::isfinite(blur[(size_t)a * bw + b])) return bail(FUSE_EINVAL);
        }
    // per-frequency factor of eq. inv, scaled by 1/(HW) for the unnormalised inverse DFT
    //   |b^(u,v)|^2 with b^ = sum_j b(j) exp(-2 pi i (u j1/H + v j2/W)),
    //   sum_{tau in W} |d^_{tau0}|^2 = sum (2 - 2 cos theta_tau) = 2|W| - 2 (Cu Cv - 1),
    //   Cu = sum_{t=-S..S} cos(2 pi u t / H)  (the sine sums vanish over the symmetric window).
    std::vector<double> fh(c->n);
    {
        const double tp = 2.0 * M_PI;
        const int rh = bh / 2, rw = bw / 2;
        std::vector<double> gr((size_t)bh * W), gi((size_t)bh * W);
        for (int a = 0; a < bh; ++a)
            for (int v = 0; v < W; ++v) {
                double sr = 0, si = 0;
                for (int b = 0; b < bw; ++b) {
                    const double ang = -tp * (double)v * (double)(b - rw) / W;
                    sr += blur[(size_t)a * bw + b] * std::cos(ang);
                    si += blur[(size_t)a * bw + b] * std::sin(ang);
                }
                gr[(size_t)a * W + v] = sr;
                gi[(size_t)a * W + v] = si;
            }
        std::vector<double> Cu(H), Cv(W);
        for (int u = 0; u < H; ++u) { double s = 0; for (int t = -S; t <= S; ++t) s += std::cos(tp * u * t / H); Cu[u] = s; }
        for (int v = 0; v < W; ++v) { double s = 0; for (int t = -S; t <= S; ++t) s += std::cos(tp * v * t / W); Cv[v] = s; }
        const double np_ = (double)c->nP;
        for (int u = 0; u < H; ++u) {
            std::vector<double> er(bh), ei(bh);
            for (int a = 0; a < bh; ++a) {
                const double ang = -tp * (double)u * (double)(a - rh) / H;
                er[a] = std::cos(ang);
                ei[a] = std::sin(ang);
            }
            for (int v = 0; v < W; ++v) {
                double br = 0, bi = 0;
                for (int a = 0; a < bh; ++a) {
                    const double xr = gr[(size_t)a * W + v], xi = gi[(size_t)a * W + v];
                    br += er[a] * xr - ei[a] * xi;
                    bi += er[a] * xi + ei[a] * xr;
                }
                const double dsum = 2.0 * c->nW - 2.0 * (Cu[u] * Cv[v] - 1.0);
                fh[(size_t)u * W + v] = 1.0 / ((1.0 + br * br + bi * bi + np_ * dsum) * (double)H * (double)W);
            }
        }
    }
    // (E E^T + rho I)^{-1} (eq. Qh_update) and F = (I + lambda1/rho E R R^T E^T)^{-1} (eq. Qm_update)
    std::vector<double> ER((size_t)Ls * Lh, 0.0);
    for (int i = 0; i < Ls; ++i)
        for (int k = 0; k < Lh; ++k) {
            double s = 0;
            for (int l = 0; l < Ll; ++l) s += Em[(size_t)i * Ll + l] * Rm[(size_t)l * Lh + k];
            ER[(size_t)i * Lh + k] = s;
        }
    std::vector<double> M1((size_t)Ls * Ls), Fm((size_t)Ls * Ls);
    const double cr = lambda1 / rho;
    for (int i = 0; i < Ls; ++i)
        for (int j = 0; j < Ls; ++j) {
            double s = 0, t = 0;
            for (int l = 0; l < Ll; ++l) s += Em[(size_t)i * Ll + l] * Em[(size_t)j * Ll + l];
            for (int k = 0; k < Lh; ++k) t += ER[(size_t)i * Lh + k] * ER[(size_t)j * Lh + k];
            M1[(size_t)i * Ls + j] = s + (i == j ? rho : 0.0);
            Fm[(size_t)i * Ls + j] = cr * t + (i == j ? 1.0 : 0.0);
        }
    if (!invert(M1, Ls) || !invert(Fm, Ls)) return bail(FUSE_EINVAL);
    // band-mixing matrices (Lin x Lout row-major)
    std::vector<double> Et((size_t)Ll * Ls), Mh((size_t)Lh * Ls), Emix(Em);
    for (int l = 0; l < Ll; ++l)
        for (int i = 0; i < Ls; ++i) Et[(size_t)l * Ls + i] = Em[(size_t)i * Ll + l];
    for (int k = 0; k < Lh; ++k)
        for (int i = 0; i < Ls; ++i) Mh[(size_t)k * Ls + i] = cr * ER[(size_t)i * Lh + k];
    // twiddles exp(-2 pi i k / N)
    auto twiddles = [&](int N) {
        std::vector<double> t(2 * (size_t)N);
        for (int k = 0; k < N; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)N;
            t[2 * (size_t)k] = std::cos(ang);
            t[2 * (size_t)k + 1] = std::sin(ang);
        }
        return t;
    };

    // ---- device buffers ----
    Sizes z = sizes_of(g, K, S, ratio, c->esz, c->wsz);
    c->sig_bytes = z.sig;
    c->plane_bytes = z.planes;
    void** imgs[] = {&c->X, &c->BX, &c->C, &c->Lam1, &c->U1, &c->Lam2, &c->U2, &c->D9b};
    for (void** p : imgs)
        if ((st = dalloc(c, p, z.img)) != FUSE_OK) return bail(st);
    if ((st = dalloc(c, &c->Y, z.cimg)) != FUSE_OK) return bail(st);
    if ((st = dalloc(c, &c->Sig, z.sig)) != FUSE_OK) return bail(st);
    if ((st = dalloc(c, &c->planes, z.planes)) != FUSE_OK) return bail(st);
    if ((st = dalloc(c, &c->omega, z.omega)) != FUSE_OK) return bail(st);
    if ((st = dalloc(c, &c->D9a, z.d9a)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->tapsT, tT)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->tapsB, tB)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->fpf, fh)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->M1, M1)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->F, Fm)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->Et, Et)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->Mh, Mh)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->Emix, Emix)) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->twH, twiddles(H))) != FUSE_OK) return bail(st);
    if ((st = upload_any(c, &c->twW, twiddles(W))) != FUSE_OK) return bail(st);
    if ((st = upload<double>(c, (void**)&c->objE, Em)) != FUSE_OK) return bail(st);
    if ((st = upload<double>(c, (void**)&c->objER, ER)) != FUSE_OK) return bail(st);
    if ((st = dalloc(c, (void**)&c->d_err, sizeof(int))) != FUSE_OK) return bail(st);
    if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return bail(FUSE_ECUDA); }
    if (!latent_tma_shape(c)) {
        c->lat_target = 128;
        c->lat_stages = 4;
        if (!latent_tma_shape(c)) c->lat_impl = 0;
    }
    const size_t nb = (c->n + 255) / 256;
    c->npartial = nb * 3 + nb * (size_t)c->nW;
    if ((st = dalloc(c, (void**)&c->partial, c->npartial * sizeof(double))) != FUSE_OK) return bail(st);
    if (c->dtype == FUSE_F64) {
        if ((st = Impl<double>::set_attrs(c)) != FUSE_OK) return bail(st);
        if ((st = Impl<double>::set_attrs_w<double>(c)) != FUSE_OK) return bail(st);
    } else {
        if ((st = Impl<float>::set_attrs(c)) != FUSE_OK) return bail(st);
        if (c->wdtype == FUSE_BF16) st = Impl<float>::set_attrs_w<__nv_bfloat16>(c);
        else st = Impl<float>::set_attrs_w<float>(c);
        if (st != FUSE_OK) return bail(st);
    }
    c->sticky = FUSE_OK;
    *out = c;
    return FUSE_OK;
}

fuse_status fuse_destroy(fuse_ctx* c) {
    if (!c) return FUSE_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
    return FUSE_OK;
}

fuse_status fuse_set_stream(fuse_ctx* c, void* stream) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    c->stream = (cudaStream_t)stream;
    return FUSE_OK;
}

fuse_status fuse_weights(fuse_ctx* c, const void* guide) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!guide) return fail(c, FUSE_EINVAL, "guide is NULL");
    return weights_impl(c, guide);
}

fuse_status fuse_set_weights(fuse_ctx* c, const void* w) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!w) return fail(c, FUSE_EINVAL, "weights pointer is NULL");
    CK(c, cudaMemcpyAsync(c->omega, w, (size_t)c->nW * c->n * c->wsz, cudaMemcpyDefault, c->stream));
    c->have_weights = true;
    return FUSE_OK;
}

fuse_status fuse_get_weights(fuse_ctx* c, void* w) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!w) return fail(c, FUSE_EINVAL, "weights pointer is NULL");
    if (!c->have_weights) return FUSE_ESTATE;
    CK(c, cudaMemcpyAsync(w, c->omega, (size_t)c->nW * c->n * c->wsz, cudaMemcpyDefault, c->stream));
    return FUSE_OK;
}

fuse_status fuse_solve(fuse_ctx* c, const void* Yl, const void* Yh, int iters, int warm, void* Xo, void* Zo) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!Yl || !Yh) return fail(c, FUSE_EINVAL, "Y_l or Y_h is NULL");
    if (iters < 0) return fail(c, FUSE_EINVAL, "iters must be >= 0");
    if (!c->have_weights) return FUSE_ESTATE;
    return solve_impl(c, Yl, Yh, iters, warm, Xo, Zo);
}

fuse_status fuse_run_host(fuse_ctx* c, const void* Yl_h, const void* Yh_h, const void* G_h, int iters, void* X_h,
                          void* Z_h) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!Yl_h || !Yh_h) return fail(c, FUSE_EINVAL, "Y_l or Y_h is NULL");
    if (iters < 0) return fail(c, FUSE_EINVAL, "iters must be >= 0");
    const size_t bl = (size_t)c->Ll * c->nl * c->esz, bhh = (size_t)c->Lh * c->n * c->esz;
    const size_t bg = (size_t)c->Lg * c->n * c->esz;
    const size_t bx = (size_t)c->Ls * c->n * c->esz, bz = (size_t)c->Ll * c->n * c->esz;
    if (!c->sYl && (st = dalloc(c, &c->sYl, bl)) != FUSE_OK) return st;
    if (!c->sYh && (st = dalloc(c, &c->sYh, bhh)) != FUSE_OK) return st;
    if (G_h && !c->sG && (st = dalloc(c, &c->sG, bg)) != FUSE_OK) return st;
    if (Z_h && !c->sZ && (st = dalloc(c, &c->sZ, bz)) != FUSE_OK) return st;
    if (X_h && !c->sX && (st = dalloc(c, &c->sX, bx)) != FUSE_OK) return st;
    CK(c, cudaMemcpyAsync(c->sYl, Yl_h, bl, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->sYh, Yh_h, bhh, cudaMemcpyHostToDevice, c->stream));
    if (G_h) {
        CK(c, cudaMemcpyAsync(c->sG, G_h, bg, cudaMemcpyHostToDevice, c->stream));
        st = weights_impl(c, c->sG);
    } else {
        if (c->Lg != c->Lh) return fail(c, FUSE_EINVAL, "guide defaults to Y_h but L_guide != L_h");
        st = weights_impl(c, c->sYh);
    }
    if (st != FUSE_OK) return st;
    st = solve_impl(c, c->sYl, c->sYh, iters, 0, X_h ? c->sX : nullptr, Z_h ? c->sZ : nullptr);
    if (st != FUSE_OK) return st;
    if (X_h) CK(c, cudaMemcpyAsync(X_h, c->sX, bx, cudaMemcpyDeviceToHost, c->stream));
    if (Z_h) CK(c, cudaMemcpyAsync(Z_h, c->sZ, bz, cudaMemcpyDeviceToHost, c->stream));
    return fuse_sync(c);
}

fuse_status fuse_objective(fuse_ctx* c, const void* Yl, const void* Yh, double out[4]) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!Yl || !Yh || !out) return fail(c, FUSE_EINVAL, "NULL argument");
    if (!c->have_x || !c->have_weights) return FUSE_ESTATE;
    return c->dtype == FUSE_F64 ? Impl<double>::objective(c, Yl, Yh, out) : Impl<float>::objective(c, Yl, Yh, out);
}

fuse_status fuse_state_bytes(fuse_ctx* c, size_t* bytes) {
    if (!c || !bytes) return FUSE_EINVAL;
    *bytes = 5 * c->n * c->Ls * c->esz + c->sig_bytes + c->plane_bytes;
    return FUSE_OK;
}

fuse_status fuse_get_state(fuse_ctx* c, void* dst) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!dst) return fail(c, FUSE_EINVAL, "NULL state buffer");
    if (!c->have_state) return FUSE_ESTATE;
    const size_t img = c->n * c->Ls * c->esz;
    char* p = (char*)dst;
    void* bufs[] = {c->Lam1, c->U1, c->Lam2, c->U2, c->X};
    for (void* b : bufs) { CK(c, cudaMemcpyAsync(p, b, img, cudaMemcpyDefault, c->stream)); p += img; }
    CK(c, cudaMemcpyAsync(p, c->Sig, c->sig_bytes, cudaMemcpyDefault, c->stream));
    p += c->sig_bytes;
    CK(c, cudaMemcpyAsync(p, c->planes, c->plane_bytes, cudaMemcpyDefault, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FUSE_OK;
}

fuse_status fuse_set_state(fuse_ctx* c, const void* src) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!src) return fail(c, FUSE_EINVAL, "NULL state buffer");
    const size_t img = c->n * c->Ls * c->esz;
    const char* p = (const char*)src;
    void* bufs[] = {c->Lam1, c->U1, c->Lam2, c->U2, c->X};
    for (void* b : bufs) { CK(c, cudaMemcpyAsync(b, p, img, cudaMemcpyDefault, c->stream)); p += img; }
    CK(c, cudaMemcpyAsync(c->Sig, p, c->sig_bytes, cudaMemcpyDefault, c->stream));
    p += c->sig_bytes;
    CK(c, cudaMemcpyAsync(c->planes, p, c->plane_bytes, cudaMemcpyDefault, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->have_state = true;
    c->have_x = true;
    return FUSE_OK;
}

fuse_status fuse_set_option(fuse_ctx* c, int option, long long value) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    switch (option) {
        case FUSE_OPT_PROFILE: c->profile = value != 0; return FUSE_OK;
        case FUSE_OPT_GRAPH: c->use_graph = value != 0; return FUSE_OK;
        case FUSE_OPT_LATENT_IMPL:
        case FUSE_OPT_LATENT_THREADS:
        case FUSE_OPT_LATENT_STAGES: {
            const int old_impl = c->lat_impl, old_t = c->lat_target, old_d = c->lat_stages;
            if (option == FUSE_OPT_LATENT_IMPL) c->lat_impl = value ? 1 : 0;
            if (option == FUSE_OPT_LATENT_THREADS) c->lat_target = (int)value;
            if (option == FUSE_OPT_LATENT_STAGES) c->lat_stages = (int)value;
            if (c->lat_target < 32 || c->lat_target > 256 || c->lat_stages < 2 || c->lat_stages > 32 ||
                !latent_tma_shape(c)) {
                c->lat_impl = old_impl; c->lat_target = old_t; c->lat_stages = old_d;
                latent_tma_shape(c);
                return fail(c, FUSE_EINVAL, "latent launch option out of range");
            }
            if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
            if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
            return FUSE_OK;
        }
        case FUSE_OPT_HALF_WINDOW: {
            const int h = value ? 1 : 0;
            if (h == c->half) return FUSE_OK;
            const size_t nWs = h ? (size_t)c->nW / 2 : (size_t)c->nW;
            const size_t bytes = nWs * c->nP * c->Ls * c->n * c->esz;
            for (auto& p : c->allocs)
                if (p == c->Sig) { CK(c, cudaStreamSynchronize(c->stream)); cudaFree(p); p = nullptr; }
            c->Sig = nullptr;
            fuse_status s2 = dalloc(c, &c->Sig, bytes);
            if (s2 != FUSE_OK) return s2;
            c->sig_bytes = bytes;
            c->half = h;
            c->have_state = false;
            c->have_x = false;
            if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
            if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
            return FUSE_OK;
        }
        case FUSE_OPT_WAIT_LIMIT:
            if (value < 1) return fail(c, FUSE_EINVAL, "wait limit must be positive");
            c->wait_limit = (unsigned)value;
            if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
            if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
            return FUSE_OK;
        default: return fail(c, FUSE_EINVAL, "unknown option");
    }
}

fuse_status fuse_profile(fuse_ctx* c, int which, double* ms, long long* launches, int reset) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    CK(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < c->ev_used; ++i) {
        float t = 0.f;
        CK(c, cudaEventElapsedTime(&t, c->ev[i].a, c->ev[i].b));
        c->latent_ms += t;
    }
    c->ev_used = 0;
    if (which == FUSE_K_LATENT) {
        if (ms) *ms = c->latent_ms;
        if (launches) *launches = c->launches_latent;
    } else if (which == FUSE_K_ALL) {
        if (ms) *ms = 0.0;
        if (launches) *launches = c->launches_all;
    } else {
        return fail(c, FUSE_EINVAL, "unknown kernel group");
    }
    if (reset) { c->latent_ms = 0.0; c->launches_latent = 0; c->launches_all = 0; }
    return FUSE_OK;
}

fuse_status fuse_sync(fuse_ctx* c) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    CK(c, cudaStreamSynchronize(c->stream));
    int flag = 0;
    CK(c, cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CK(c, cudaMemset(c->d_err, 0, sizeof(int)));
        return fail(c, FUSE_ETIMEOUT, "a bounded device-side barrier wait gave up");
    }
    return FUSE_OK;
}

fuse_status fuse_selftest(fuse_ctx* c, int which) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (which != 1) return fail(c, FUSE_EINVAL, "unknown self-test");
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    wait_selftest_kernel<<<1, 32, 0, c->stream>>>(c->d_err, 1000u, 2);
    c->launches_all++;
    CKL(c, "wait_selftest_kernel");
    CK(c, cudaStreamSynchronize(c->stream));
    int flag = 0;
    CK(c, cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    CK(c, cudaMemset(c->d_err, 0, sizeof(int)));
    if (flag != 2) return fail(c, FUSE_ECUDA, "bounded wait did not report its timeout");
    return FUSE_OK;
}

const char* fuse_last_error(const fuse_ctx* c) { return c ? c->err.c_str() : ""; }

fuse_status fuse_reset_error(fuse_ctx* c) {
    if (!c) return FUSE_EINVAL;
    c->sticky = FUSE_OK;
    c->err.clear();
    return FUSE_OK;
}

}  // extern "C"
