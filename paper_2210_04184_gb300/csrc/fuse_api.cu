// C-ABI of the NLPR multiband-fusion solver: context, host FP64 set-up, launch sequence.
// The contract of every entry point is in include/fuse.h.
#include "fuse.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.cuh"
#include "dispatch.cuh"
#include "k_fft.cuh"
#include "k_grad.cuh"
#include "k_latent.cuh"
#include "k_monitor.cuh"
#include "k_objective.cuh"
#include "k_pixel.cuh"
#include "k_stencil.cuh"
#include "k_weights.cuh"
#include "launch.cuh"

using namespace fuse;

namespace fuse {

// Self-check of the bounded-wait machinery: waits on a barrier that nothing ever completes.
// The wait must give up after `limit` polls and set bit `code` in *err.
__global__ void wait_selftest_kernel(int* err, unsigned limit, int code) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0u, limit, err, code);
}

}  // namespace fuse

namespace {

constexpr int kMaxSmem = 200 * 1024;
// blocks of the grid-stride reduction kernels of the residual monitor (a fixed count, so the sums
// are formed in the same order on every device)
constexpr int kMonBlocks = 608;
// SM count assumed where no device is queried (fuse_workspace_bytes: the sizes do not depend on it)
constexpr int kDefaultSMs = 152;

struct Event2 { cudaEvent_t a, b; };

// Iterations captured in one CUDA graph: a solve of up to this many iterations replays one graph;
// longer solves replay full graphs and one for the remainder.
constexpr int kGraphIters = 256;

// A captured loop of `len` iterations; `cold` marks a loop whose first latent pass reads no state
// (it starts a solve from zero).  Two are cached per context or batch (the full loop and the
// remainder of a long solve), the least recently used one is replaced.
struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
    int len = 0, cold = 0;
    long long launches = 0;
    unsigned long long used = 0;
};

struct LoopCache {
    LoopGraph g[2];
    unsigned long long tick = 0;
    LoopGraph* find(int len, int cold) {
        for (LoopGraph& x : g)
            if (x.exec && x.len == len && x.cold == cold) { x.used = ++tick; return &x; }
        return nullptr;
    }
    LoopGraph* victim() { return g[0].used <= g[1].used ? &g[0] : &g[1]; }
    void clear() {
        for (LoopGraph& x : g) {
            if (x.exec) cudaGraphExecDestroy(x.exec);
            x = LoopGraph{};
        }
    }
};

}  // namespace

struct GradWork;

// Second capture stream of a captured iteration loop: B X and the pixel updates of an iteration
// need only X, like the latent pass, so in a captured loop they run on this stream beside the
// latent pass (fork after the inverse DFT); the next iteration's right-hand side, which reads
// their U1 and U2, waits for them (join).
struct SideBranch {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    bool create() {
        return cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess;
    }
    void destroy() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (s) cudaStreamDestroy(s);
        s = nullptr;
        fork = join = nullptr;
    }
};

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
    SideBranch side;
    int device = 0, nsm = kDefaultSMs;      // device and its SM count (launch-shape heuristics)
    // launch shapes
    int vec = 4, lat_Ty = 1, lat_threads = 0;
    size_t lat_smem = 0;
    int w_Ty = 1;
    size_t w_smem = 0;
    int fr_tpr = 32, fr_rpb = 1, fc_cw = 8, fc_tpc = 32;
    size_t fr_smem = 0, fc_smem = 0, st_smem = 0, px_smem = 0;
    int px_threads = 128;
    FFTPlan planH{}, planW{};
    // DFT solve: 1 = register-resident passes (k_wfft.cuh; sides 32 P), 0 = shared-memory
    // Stockham passes; fT: f in the register form's spectrum order (NULL when not eligible)
    int fft_impl = 0;
    void* fT = nullptr;
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
    LoopCache loops;
    int fault_alloc = -1, alloc_count = 0;
    // latent pass variant: 0 = register-staged loads, 1 = bulk-copy (TMA) ring
    int lat_impl = 1, lat_target = 128, lat_stages = 6, lat_bpb = 1;
    int lt_Ty = 1, lt_ncons = 0;
    size_t lt_smem = 0;
    int* d_err = nullptr;
    unsigned wait_limit = 1u << 22;
    // half-window latent state (one offset of each +-tau pair); 0 = full window
    int half = 1;
    // latent state storage: 0 = the iterate type, 1 = 16-bit fixed point relative to mu
    int sfmt = 0;
    // sampling mask [H][W] (uint8, ratio 1) replacing the regular lattice; NULL = lattice.
    // The buffer (mask_buf) is kept once allocated, so launch arguments taken earlier (a batch)
    // never point to freed memory.
    void *mask = nullptr, *mask_buf = nullptr;
    // reverse pass: workspace, iterations per checkpointed segment (0 = one segment), a counter
    // bumped by every call that changes inputs or state (a taped forward is valid while unchanged)
    GradWork* gw = nullptr;
    int grad_seg = 0, grad_weights = 0;
    long long epoch = 0;
    // host FP64 copies of (E E^T + rho I)^{-1}, F and E R, for the parameter derivatives
    std::vector<double> hM1, hF, hER;
    // spectral condition numbers of A (eq. inv), E E^T + rho I and F^{-1} (fuse_conditioning)
    double cond[3] = {0.0, 0.0, 0.0};
    // host copies of the blur taps (b for B^T, flipped b for B) for the square-blur stencil, and
    // their factors cu (bh values) then cv when the taps are separable (empty otherwise)
    std::vector<double> htapsT, htapsB, hsepT, hsepB;
    int sep_blur = 1;           // FUSE_OPT_SEPARABLE_BLUR
    // latent state read / written by the next latent launch (NULL = Sig, in place); set only
    // around directly launched iterations of the taped forward, never while capturing
    void *lat_in = nullptr, *lat_out = nullptr;
    // X update: 0 = the paper's splitting, 1 = S B kept in the X system (per-alias-class solve).
    // E E^T = eet_eps I up to the relative deviation eet_dev (measured at fuse_init); the class
    // tables (sbq, sbp, sbk) and the column-pass shape (fa_m base columns per block, fa_tpc
    // threads per column) are set when the variant is first selected.
    int xmode = 0;
    double eet_eps = 0.0, eet_dev = 0.0;
    void *sbq = nullptr, *sbp = nullptr, *sbk = nullptr;
    int fa_m = 1, fa_tpc = 32;
    size_t fa_smem = 0;
    // residual monitor (FUSE_OPT_RESIDUALS): copies of Lambda1, U1, Lambda2, U2 and of the adjoint
    // planes entering the last iteration of a solve, the monitoring latent pass's planes, FP64
    // block sums ([latent blocks (room for mon_lat_cap)] [pixel pass] [dual image]); mon_epoch: the
    // context epoch of the last monitored iteration, mon_lat: its latent block count
    int monitor = 0;
    void *mL1 = nullptr, *mU1 = nullptr, *mL2 = nullptr, *mU2 = nullptr, *mPo = nullptr, *mPm = nullptr;
    double* mon_part = nullptr;
    size_t mon_lat_cap = 0, mon_lat = 0;
    long long mon_epoch = -1;
};

namespace {
inline void* lat_src(const fuse_ctx* c) { return c->lat_in ? c->lat_in : c->Sig; }
inline void* lat_dst(const fuse_ctx* c) { return c->lat_out ? c->lat_out : c->Sig; }
// The captured iteration loops depend on the launch configuration: dropped whenever it changes.
inline void drop_graphs(fuse_ctx* c) { c->loops.clear(); }
}  // namespace

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
// Extreme eigenvalues of the symmetric n x n matrix A (cyclic Jacobi rotations until the
// off-diagonal part is negligible).
void sym_eig_range(std::vector<double> A, int n, double* lo, double* hi) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += A[(size_t)i * n + i] * A[(size_t)i * n + i];
            for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        }
        if (off <= 1e-30 * diag) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double th = 0.5 * (aqq - app) / apq;
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {                       // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = cs * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {                       // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = cs * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
            }
    }
    *lo = *hi = A[0];
    for (int i = 1; i < n; ++i) {
        *lo = std::min(*lo, A[(size_t)i * n + i]);
        *hi = std::max(*hi, A[(size_t)i * n + i]);
    }
}

// Factors of a separable square blur: taps(u, v) = cu[u] cv[v] up to rounding (1e-13 of the
// largest tap), returned as cu[0..b) then cv[0..b); empty when the taps are not of rank one.
std::vector<double> separable_factors(const std::vector<double>& t, int b) {
    int am = 0, bm = 0;
    double mx = 0.0;
    for (int u = 0; u < b; ++u)
        for (int v = 0; v < b; ++v)
            if (std::fabs(t[(size_t)u * b + v]) > mx) { mx = std::fabs(t[(size_t)u * b + v]); am = u; bm = v; }
    if (mx == 0.0) return {};
    std::vector<double> f(2 * (size_t)b);
    for (int u = 0; u < b; ++u) f[u] = t[(size_t)u * b + bm];
    for (int v = 0; v < b; ++v) f[b + v] = t[(size_t)am * b + v] / t[(size_t)am * b + bm];
    for (int u = 0; u < b; ++u)
        for (int v = 0; v < b; ++v)
            if (std::fabs(t[(size_t)u * b + v] - f[u] * f[b + v]) > 1e-13 * mx) return {};
    return f;
}

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

// Validates the problem and picks the default launch shapes for a device with `nsm` SMs.
fuse_status check_geometry(fuse_ctx* c, const fuse_geometry* g, int K, int S, int ratio, fuse_dtype dtype,
                           fuse_dtype wdtype, int bh, int bw, Shapes* sh, FFTPlan* pH, FFTPlan* pW,
                           int nsm = kDefaultSMs) {
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
    // small images: fewer rows per block until the pass has about two blocks per SM
    const int npair_ = (g->L_s + 1) / 2;
    while (sh->fr_rpb > 1 && (long long)((g->H + sh->fr_rpb - 1) / sh->fr_rpb) * npair_ < 2 * nsm) sh->fr_rpb /= 2;
    sh->fr_smem = 2 * (size_t)sh->fr_rpb * g->W * csz;
    if (sh->fr_smem > kMaxSmem) return fail(c, FUSE_EUNSUPPORTED, "W too large for the FFT");
    // fft columns
    sh->fc_cw = dtype == FUSE_F64 ? 4 : 8;
    while (sh->fc_cw > 1 && (size_t)sh->fc_cw * (2 * g->H + 1) * csz > kMaxSmem) sh->fc_cw /= 2;
    // narrower blocks until the pass has about four blocks per SM (one wave at four resident
    // blocks: a column block holds 256 threads and tens of KB of shared memory)
    while (sh->fc_cw > 2 && (long long)((g->W + sh->fc_cw - 1) / sh->fc_cw) * npair_ < 4 * nsm) sh->fc_cw /= 2;
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
// rows, 32 bytes of pixels per thread), `stages` ring slots; false if W is not a multiple of
// the vector or the ring does not fit in shared memory (the register-staged pass is used then).
bool latent_tma_shape(fuse_ctx* c) {
    const int tvec = (int)(32 / c->esz);        // 8 floats or 4 doubles per thread and chunk
    if (c->W % tvec) return false;
    const int tpr = c->W / tvec;
    int Ty = c->lat_target / tpr;
    if (Ty < 1) Ty = 1;
    if (Ty > c->H) Ty = c->H;
    while (Ty > 1 && ((tpr * Ty + 31) / 32) * 32 + 32 > 288) --Ty;
    const int ncons = ((tpr * Ty + 31) / 32) * 32;
    if (ncons + 32 > 288) return false;
    const size_t ssz = c->sfmt ? 2 : c->esz;     // bytes of one stored state element
    // ring, the tiles Xo, Vs, two H tiles and Xs (see latent_tma_body), mbarriers
    const size_t smem = (size_t)c->lat_stages * Ty * c->W * ssz + 5 * (size_t)Ty * c->W * c->esz +
                        2 * (size_t)c->lat_stages * 8;
    if (smem > (size_t)kMaxSmem || c->lat_stages < 1) return false;
    c->lt_Ty = Ty;
    c->lt_ncons = ncons;
    c->lt_smem = smem;
    return true;
}

// Dynamic shared-memory cap of the monitoring latent kernels of this context's types.
bool set_monitor_smem(fuse_ctx* c) {
    cudaError_t e;
    if (c->dtype == FUSE_F64) e = latent_set_smem<double, double>(c->K, kMaxSmem);
    else if (c->wdtype == FUSE_BF16) e = latent_set_smem<float, __nv_bfloat16>(c->K, kMaxSmem);
    else e = latent_set_smem<float, float>(c->K, kMaxSmem);
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// typed launch sequence
// ---------------------------------------------------------------------------------------

template <typename T>
struct Impl {

    // ---- argument blocks of the iteration kernels ----
    static StencilArgs<T> st_args(fuse_ctx* c, const void* in, void* out, const void* taps) {
        return StencilArgs<T>{(const T*)in, (T*)out, (const T*)taps, c->bw, c->H, c->W,
                              (const T*)c->U2, (const T*)c->planes, c->S, c->half};
    }
    static FFTArgs<T> fft_args(fuse_ctx* c, int rpb, int cw) {
        return FFTArgs<T>{(const T*)c->C, (cplx<T>*)c->Y, (T*)c->X, (const T*)c->fpf, c->H, c->W, c->Ls,
                          c->planW, c->planH, (const cplx<T>*)c->twW, (const cplx<T>*)c->twH, rpb, cw,
                          c->fft_impl == 1 ? (const T*)c->fT : nullptr};
    }
    static PixelArgs<T> px_args(fuse_ctx* c) {
        return PixelArgs<T>{(const T*)c->X, (const T*)c->BX, (T*)c->Lam1, (T*)c->U1, (T*)c->Lam2, (T*)c->U2,
                            (const T*)c->D9a, (const T*)c->D9b, (const T*)c->M1, (const T*)c->F,
                            c->H, c->W, c->Ls, c->d, (T)c->rho, (const uint8_t*)c->mask, c->xmode == 1 ? 1 : 0};
    }
    template <typename WT>
    static LatentArgs<T, WT> lat_args(fuse_ctx* c, int Ty, int ncons, int D, int bpb, int zero_in = 0) {
        return LatentArgs<T, WT>{(const T*)c->X, (const WT*)c->omega, (const T*)lat_src(c), (T*)lat_dst(c),
                                 (T*)c->planes, c->H, c->W,
                                 c->Ls, c->S, Ty, ncons, D, (T)(c->lam2 / c->rho), c->d_err, c->wait_limit,
                                 c->half, bpb, zero_in};
    }

    static fuse_status set_attrs(fuse_ctx* c) {
        const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        // The cap is a property of the kernel function shared by every context in the process,
        // so it is set to the largest size any context may request, never to this context's.
        CK(c, cudaFuncSetAttribute(fft_rows_fwd_kernel<T>, A, kMaxSmem));
        CK(c, cudaFuncSetAttribute(fft_rows_inv_kernel<T>, A, kMaxSmem));
        CK(c, cudaFuncSetAttribute(fft_cols_kernel<T>, A, kMaxSmem));
        CK(c, cudaFuncSetAttribute(fft_cols_alias_kernel<T>, A, kMaxSmem));
        CK(c, wfft_set_smem<T>(kMaxSmem));
        CK(c, pixel_stencil_set_smem<T>(c->bh, kMaxSmem));
        CK(c, cudaFuncSetAttribute(band_mix_kernel<T>, A, kMaxSmem));
        return FUSE_OK;
    }

    template <typename WT>
    static fuse_status set_attrs_w(fuse_ctx* c) {
        const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        CK(c, cudaFuncSetAttribute(weights_kernel<T, WT>, A, kMaxSmem));
        CK(c, (latent_set_smem<T, WT>(c->K, kMaxSmem)));
        return FUSE_OK;
    }

    // Launches a blur stencil: the square-blur kernel (taps in the argument space) when
    // bh == bw, else the generic one (taps in shared memory).
    template <int MODE>
    static void stencil_launch(fuse_ctx* c, cudaStream_t s, const StencilArgs<T>& a) {
        dim3 grid((unsigned)((c->W + ST_TX - 1) / ST_TX), (unsigned)((c->H + ST_TY - 1) / ST_TY), (unsigned)c->Ls);
        const double *ht = nullptr, *sep = nullptr;
        if (c->bh == c->bw) {
            const bool isB = a.taps == (const T*)c->tapsB;
            ht = isB ? c->htapsB.data() : c->htapsT.data();
            const std::vector<double>& f = isB ? c->hsepB : c->hsepT;
            if (c->sep_blur && !f.empty() && c->W % 4 == 0) sep = f.data();     // four-column vectors
        }
        fuse::stencil_launch<T, MODE>(a, c->bh, sep, ht, grid, c->st_smem, s);
    }

    // MODE 0: out = B in (taps = flipped b); MODE 1: C = B^T U1 + U2 + R (taps = b).
    template <int MODE>
    static void stencil(fuse_ctx* c, cudaStream_t s, const void* in, void* out, const void* taps) {
        stencil_launch<MODE>(c, s, st_args(c, in, out, taps));
    }

    static void pixel(fuse_ctx* c, cudaStream_t s) {
        const unsigned pblocks = (unsigned)((c->n + c->px_threads - 1) / c->px_threads);
        pixel_launch<T>(px_args(c), pblocks, (unsigned)c->px_threads, c->px_smem, s);
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

    // zero_in: the state entering this pass is zero (the first iteration of a cold solve); the
    // bulk-copy pass then reads none of it.  The register-staged pass always reads it.
    template <typename WT>
    static void latent(fuse_ctx* c, cudaStream_t s, bool zero_in) {
        const unsigned rowsW = (unsigned)(c->half ? c->S + 1 : 2 * c->S + 1);
        if (c->lat_impl == 1) {
            dim3 grid((unsigned)((c->H + c->lt_Ty - 1) / c->lt_Ty), (unsigned)((c->Ls + c->lat_bpb - 1) / c->lat_bpb),
                      rowsW);
            const LatentArgs<T, WT> a = lat_args<WT>(c, c->lt_Ty, c->lt_ncons, c->lat_stages, c->lat_bpb, zero_in);
            latent_tma_launch<T, WT>(a, c->K, c->sfmt == 1, grid, (unsigned)(c->lt_ncons + 32), c->lt_smem, s);
            return;
        }
        dim3 grid((unsigned)((c->H + c->lat_Ty - 1) / c->lat_Ty), (unsigned)c->Ls, rowsW);
        latent_reg_launch<T, WT>((const T*)c->X, (const WT*)c->omega, (const T*)lat_src(c), (T*)lat_dst(c),
                                 (T*)c->planes, c->H, c->W, c->Ls, c->S, c->lat_Ty, (T)(c->lam2 / c->rho), c->half,
                                 c->K, grid, (unsigned)c->lat_threads, c->lat_smem, s);
    }

    static void latent_any(fuse_ctx* c, cudaStream_t s, bool zero_in);

    // The monitoring latent pass (bulk-copy kernel, state in the iterate type) and the residual
    // sums of the iteration that ran it (k_monitor.cuh).
    template <typename WT>
    static void latent_monitor(fuse_ctx* c, cudaStream_t s, bool zero_in) {
        const unsigned rowsW = (unsigned)(c->half ? c->S + 1 : 2 * c->S + 1);
        dim3 grid((unsigned)((c->H + c->lt_Ty - 1) / c->lt_Ty), (unsigned)((c->Ls + c->lat_bpb - 1) / c->lat_bpb),
                  rowsW);
        LatentArgs<T, WT> a = lat_args<WT>(c, c->lt_Ty, c->lt_ncons, c->lat_stages, c->lat_bpb, zero_in);
        a.mplanes = (T*)c->mPm;
        a.mpart = c->mon_part;
        c->mon_lat = (size_t)grid.x * grid.y * grid.z;
        const size_t smem = c->lt_smem + 2 * (size_t)c->lt_Ty * c->W * sizeof(T);     // two more tiles
        latent_monitor_launch<T, WT>(a, c->K, grid, (unsigned)(c->lt_ncons + 32), smem, s);
    }

    static fuse_status monitor_sums(fuse_ctx* c, cudaStream_t s) {
        const size_t cnt = c->n * c->Ls;
        double* pix = c->mon_part + c->mon_lat_cap;
        monitor_pixel_kernel<T><<<kMonBlocks, 256, 0, s>>>((const T*)c->Lam1, (const T*)c->U1, (const T*)c->Lam2,
                                                           (const T*)c->U2, (const T*)c->mL1, (T*)c->mU1,
                                                           (const T*)c->mL2, (T*)c->mU2, cnt, pix);
        CKL(c, "monitor_pixel_kernel");
        sub_kernel<T><<<kMonBlocks, 256, 0, s>>>((T*)c->mPm, (const T*)c->mPo, c->plane_bytes / sizeof(T));
        CKL(c, "sub_kernel");
        // B^T dP1 + dP2 + sum D^T dQ into C (free until the next iteration forms it)
        const StencilArgs<T> a{(const T*)c->mU1, (T*)c->C, (const T*)c->tapsT, c->bw, c->H, c->W,
                               (const T*)c->mU2, (const T*)c->mPm, c->S, c->half};
        stencil_launch<1>(c, s, a);
        CKL(c, "stencil_kernel (dual residual)");
        sumsq_kernel<T><<<kMonBlocks, 256, 0, s>>>((const T*)c->C, cnt, pix + kMonBlocks);
        CKL(c, "sumsq_kernel");
        c->launches_all += 4;
        return FUSE_OK;
    }

    // One ADMM iteration (Sec. IV): C, X update, P1/P2/duals, latent pass.  With xmode 1 (S B
    // kept in the X system): C = G + U2 + R with the fixed data term G in U1, the column pass
    // solves the alias classes, and there is no B X and no P1.  zero_in: see latent().
    // side (captured loops): B X and the pixel pass run on c->side.s beside the latent pass;
    // join_prev: wait for the previous iteration's side branch before the right-hand side.
    static fuse_status iterate(fuse_ctx* c, cudaStream_t s, bool timed, bool zero_in = false, bool monitor = false,
                               bool side = false, bool join_prev = false) {
        if (side && join_prev) CK(c, cudaStreamWaitEvent(s, c->side.join, 0));
        if (c->xmode == 1) {
            dim3 grid((unsigned)((c->W + ST_TX - 1) / ST_TX), (unsigned)((c->H + ST_TY - 1) / ST_TY), (unsigned)c->Ls);
            rhs_sum_kernel<T><<<grid, dim3(ST_TX, ST_BY), 0, s>>>(st_args(c, c->U1, c->C, nullptr));
            CKL(c, "rhs_sum_kernel");
        } else {
            stencil<1>(c, s, c->U1, c->C, c->tapsT);
            CKL(c, "stencil_kernel (right-hand side)");
        }
        const FFTArgs<T> fa = fft_args(c, c->fr_rpb, c->fc_cw);
        if (c->xmode == 1) {
            dim3 rgrid((unsigned)((c->H + c->fr_rpb - 1) / c->fr_rpb), (unsigned)c->npair);
            fft_rows_fwd_kernel<T><<<rgrid, c->fr_tpr * c->fr_rpb, c->fr_smem, s>>>(fa);
            CKL(c, "fft_rows_fwd_kernel");
            const FFTAliasArgs<T> aa{(cplx<T>*)c->Y, c->H, c->W, c->d, c->fa_m, c->planH, (const cplx<T>*)c->twH,
                                     (const T*)c->sbq, (const cplx<T>*)c->sbp, (const T*)c->sbk};
            const int w = c->W / c->d;
            dim3 agrid((unsigned)((w + c->fa_m - 1) / c->fa_m), (unsigned)c->npair);
            fft_cols_alias_kernel<T><<<agrid, c->fa_m * c->d * c->fa_tpc, c->fa_smem, s>>>(aa);
            CKL(c, "fft_cols_alias_kernel");
            fft_rows_inv_kernel<T><<<rgrid, c->fr_tpr * c->fr_rpb, c->fr_smem, s>>>(fa);
            CKL(c, "fft_rows_inv_kernel");
        } else {
            const fuse_status st = dft_solve(c, s, fa);
            if (st != FUSE_OK) return st;
        }
        cudaStream_t sp = s;
        if (side) {
            CK(c, cudaEventRecord(c->side.fork, s));
            CK(c, cudaStreamWaitEvent(c->side.s, c->side.fork, 0));
            sp = c->side.s;
        }
        if (c->xmode != 1) {
            stencil<0>(c, sp, c->X, c->BX, c->tapsB);
            CKL(c, "stencil_kernel (B X)");
        }
        pixel(c, sp);
        CKL(c, "pixel_kernel");
        if (side) CK(c, cudaEventRecord(c->side.join, c->side.s));
        if (timed) {
            if (c->ev_used == c->ev.size()) {
                Event2 e{};
                CK(c, cudaEventCreate(&e.a));
                CK(c, cudaEventCreate(&e.b));
                c->ev.push_back(e);
            }
            Event2& e = c->ev[c->ev_used++];
            CK(c, cudaEventRecord(e.a, s));
            latent_any(c, s, zero_in);
            CK(c, cudaEventRecord(e.b, s));
        } else if (monitor) {
            if constexpr (sizeof(T) == 8) {
                latent_monitor<double>(c, s, zero_in);
            } else {
                if (c->wdtype == FUSE_BF16) latent_monitor<__nv_bfloat16>(c, s, zero_in);
                else latent_monitor<float>(c, s, zero_in);
            }
        } else {
            latent_any(c, s, zero_in);
        }
        CKL(c, "latent kernel");
        if (monitor) return monitor_sums(c, s);
        return FUSE_OK;
    }

    // out = A^{-1} in (eq. inv) with the plain factor f: three DFT passes over fa (input fa.C,
    // output fa.X), in the register-resident form when the context selected it.
    static fuse_status dft_solve(fuse_ctx* c, cudaStream_t s, const FFTArgs<T>& fa) {
        if (c->fft_impl == 1) {
            const size_t smem = wfft_cols_smem<T>(c->H);
            wfft_pass_launch<T>(fa, 0, c->npair, 0, s);
            CKL(c, "wfft_rows_fwd_kernel");
            wfft_pass_launch<T>(fa, 1, c->npair, smem, s);
            CKL(c, "wfft_cols_kernel");
            wfft_pass_launch<T>(fa, 2, c->npair, 0, s);
            CKL(c, "wfft_rows_inv_kernel");
            return FUSE_OK;
        }
        dim3 rgrid((unsigned)((c->H + c->fr_rpb - 1) / c->fr_rpb), (unsigned)c->npair);
        fft_rows_fwd_kernel<T><<<rgrid, c->fr_tpr * c->fr_rpb, c->fr_smem, s>>>(fa);
        CKL(c, "fft_rows_fwd_kernel");
        dim3 cgrid((unsigned)((c->W + c->fc_cw - 1) / c->fc_cw), (unsigned)c->npair);
        fft_cols_kernel<T><<<cgrid, c->fc_cw * c->fc_tpc, c->fc_smem, s>>>(fa);
        CKL(c, "fft_cols_kernel");
        fft_rows_inv_kernel<T><<<rgrid, c->fr_tpr * c->fr_rpb, c->fr_smem, s>>>(fa);
        CKL(c, "fft_rows_inv_kernel");
        return FUSE_OK;
    }

    static fuse_status objective(fuse_ctx* c, const void* Yl, const void* Yh, double out[4]);

    static fuse_status sb_data_term(fuse_ctx* c, cudaStream_t s) {
        const size_t tot = c->n * c->Ls;
        upsample_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const T*)c->D9a, (T*)c->BX, c->H, c->W, c->d,
                                                                         c->Ls, (T)(1.0 / c->rho));
        CKL(c, "upsample_kernel");
        stencil<0>(c, s, c->BX, c->U1, c->tapsT);
        CKL(c, "stencil_kernel (B^T S^T Y_l E^T)");
        c->launches_all += 2;
        return FUSE_OK;
    }
};

template <typename T>
void Impl<T>::latent_any(fuse_ctx* c, cudaStream_t s, bool zero_in) {
    if constexpr (sizeof(T) == 8) {
        latent<double>(c, s, zero_in);
    } else {
        if (c->wdtype == FUSE_BF16) latent<__nv_bfloat16>(c, s, zero_in);
        else latent<float>(c, s, zero_in);
    }
}

template <typename T>
fuse_status Impl<T>::objective(fuse_ctx* c, const void* Yl, const void* Yh, double out[4]) {
    const size_t n = c->n;
    stencil<0>(c, c->stream, c->X, c->BX, c->tapsB);
    const unsigned nb = (unsigned)((n + 255) / 256);
    obj_data_kernel<T><<<nb, 256, 0, c->stream>>>((const T*)c->X, (const T*)c->BX, (const T*)Yl, (const T*)Yh,
                                                   c->objE, c->objER, c->H, c->W, c->d, c->Ls, c->Ll, c->Lh,
                                                   c->partial, (const uint8_t*)c->mask);
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

// Zero ADMM state.  clear_sigma = false leaves the latent state as it is: the caller's next
// iteration then runs a latent pass that reads none of it (zero_in) and overwrites all of it.
fuse_status zero_state(fuse_ctx* c, cudaStream_t s, bool clear_sigma = true) {
    const size_t img = c->n * c->Ls * c->esz;
    CK(c, cudaMemsetAsync(c->Lam1, 0, img, s));
    CK(c, cudaMemsetAsync(c->U1, 0, img, s));
    CK(c, cudaMemsetAsync(c->Lam2, 0, img, s));
    CK(c, cudaMemsetAsync(c->U2, 0, img, s));
    CK(c, cudaMemsetAsync(c->X, 0, img, s));
    if (clear_sigma) CK(c, cudaMemsetAsync(c->Sig, 0, c->sig_bytes, s));
    CK(c, cudaMemsetAsync(c->planes, 0, c->plane_bytes, s));
    return FUSE_OK;
}

// kernels launched by one iteration (Impl::iterate)
int iteration_launches(const fuse_ctx* c) { return c->xmode == 1 ? 6 : 7; }

// Replays `len` iterations from one captured graph (captured on first use; `cold`: the first
// iteration's latent pass reads no state).
fuse_status launch_loop(fuse_ctx* c, int len, bool cold) {
    LoopGraph* lg = c->loops.find(len, cold);
    if (!lg) {
        const bool f64 = c->dtype == FUSE_F64;
        CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        fuse_status st = FUSE_OK;
        int forked = 0;
        for (int t = 0; t < len && st == FUSE_OK; ++t, ++forked)
            st = f64 ? Impl<double>::iterate(c, c->cap_stream, false, cold && t == 0, false, true, t > 0)
                     : Impl<float>::iterate(c, c->cap_stream, false, cold && t == 0, false, true, t > 0);
        // the side branch of the last iteration joins the loop's stream before the capture ends
        if (forked && cudaStreamWaitEvent(c->cap_stream, c->side.join, 0) != cudaSuccess && st == FUSE_OK)
            st = fail(c, FUSE_ECUDA, "cudaStreamWaitEvent");
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (st != FUSE_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return fail_cuda(c, "cudaStreamEndCapture", e);
        lg = c->loops.victim();
        if (lg->exec) cudaGraphExecDestroy(lg->exec);
        *lg = LoopGraph{};
        e = cudaGraphInstantiate(&lg->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { lg->exec = nullptr; return fail_cuda(c, "cudaGraphInstantiate", e); }
        lg->len = len;
        lg->cold = cold;
        lg->launches = (long long)len * iteration_launches(c);
        lg->used = ++c->loops.tick;
    }
    CK(c, cudaGraphLaunch(lg->exec, c->stream));
    c->launches_all += lg->launches;
    c->launches_latent += len;
    return FUSE_OK;
}

// Runs `iters` iterations: the whole loop replayed from captured graphs of up to kGraphIters
// iterations, or launched directly when profiling or with graphs switched off.  cold: the state
// entering the first iteration is zero and its latent pass reads none of it.
fuse_status run_iterations_plain(fuse_ctx* c, int iters, bool cold);

// The last iteration of a monitored solve: the entering Lambda1, U1, Lambda2, U2 and adjoint
// planes are copied aside, then the iteration runs with the monitoring latent pass and the
// residual sums (directly launched).
fuse_status monitored_iteration(fuse_ctx* c, bool zero_in) {
    if (c->lat_impl != 1 || c->sfmt != 0 || c->xmode != 0)
        return fail(c, FUSE_EUNSUPPORTED, "the residual monitor needs the bulk-copy latent pass, the state in the "
                                          "iterate type and the paper's splitting");
    if (c->lt_smem + 2 * (size_t)c->lt_Ty * c->W * c->esz > (size_t)kMaxSmem)
        return fail(c, FUSE_EUNSUPPORTED, "the monitoring latent pass does not fit shared memory");
    const size_t img = c->n * c->Ls * c->esz;
    cudaStream_t s = c->stream;
    CK(c, cudaMemcpyAsync(c->mL1, c->Lam1, img, cudaMemcpyDeviceToDevice, s));
    CK(c, cudaMemcpyAsync(c->mU1, c->U1, img, cudaMemcpyDeviceToDevice, s));
    CK(c, cudaMemcpyAsync(c->mL2, c->Lam2, img, cudaMemcpyDeviceToDevice, s));
    CK(c, cudaMemcpyAsync(c->mU2, c->U2, img, cudaMemcpyDeviceToDevice, s));
    CK(c, cudaMemcpyAsync(c->mPo, c->planes, c->plane_bytes, cudaMemcpyDeviceToDevice, s));
    fuse_status st = c->dtype == FUSE_F64 ? Impl<double>::iterate(c, s, false, zero_in, true)
                                          : Impl<float>::iterate(c, s, false, zero_in, true);
    if (st != FUSE_OK) return st;
    c->launches_all += iteration_launches(c);
    c->launches_latent += 1;
    return FUSE_OK;
}

fuse_status run_iterations(fuse_ctx* c, int iters, bool cold = false) {
    if (iters <= 0 || !c->monitor) return run_iterations_plain(c, iters, cold);
    fuse_status st = run_iterations_plain(c, iters - 1, cold);
    if (st != FUSE_OK) return st;
    return monitored_iteration(c, cold && iters == 1);
}

fuse_status run_iterations_plain(fuse_ctx* c, int iters, bool cold) {
    if (iters <= 0) return FUSE_OK;
    const bool f64 = c->dtype == FUSE_F64;
    if (c->profile || !c->use_graph) {
        for (int t = 0; t < iters; ++t) {
            fuse_status st = f64 ? Impl<double>::iterate(c, c->stream, c->profile, cold && t == 0)
                                 : Impl<float>::iterate(c, c->stream, c->profile, cold && t == 0);
            if (st != FUSE_OK) return st;
            c->launches_all += iteration_launches(c);
            c->launches_latent += 1;
        }
        return FUSE_OK;
    }
    for (int done = 0; done < iters;) {
        const int len = std::min(iters - done, kGraphIters);
        fuse_status st = launch_loop(c, len, cold && done == 0);
        if (st != FUSE_OK) return st;
        done += len;
    }
    return FUSE_OK;
}

fuse_status solve_impl(fuse_ctx* c, const void* Yl, const void* Yh, int iters, int warm, void* Xo, void* Zo) {
    const bool f64 = c->dtype == FUSE_F64;
    fuse_status st;
    ++c->epoch;
    // S^T Y_l E^T on the sampled lattice and lambda1/rho Y_h R^T E^T (eqs. Qh_update, Qm_update)
    st = f64 ? Impl<double>::band_mix(c, c->stream, Yl, c->D9a, c->Et, c->nl, c->Ll, c->Ls)
             : Impl<float>::band_mix(c, c->stream, Yl, c->D9a, c->Et, c->nl, c->Ll, c->Ls);
    if (st != FUSE_OK) return st;
    st = f64 ? Impl<double>::band_mix(c, c->stream, Yh, c->D9b, c->Mh, c->n, c->Lh, c->Ls)
             : Impl<float>::band_mix(c, c->stream, Yh, c->D9b, c->Mh, c->n, c->Lh, c->Ls);
    if (st != FUSE_OK) return st;
    // A cold start with at least one iteration leaves the latent state uncleared: the first
    // latent pass of the bulk-copy kernel takes it as zero and overwrites every entry.
    bool cold = false;
    if (!warm || !c->have_state) {
        cold = iters > 0 && c->lat_impl == 1;
        st = zero_state(c, c->stream, !cold);
        if (st != FUSE_OK) return st;
        c->have_state = true;
    }
    if (c->xmode == 1) {
        // the fixed data term of the variant: U1 = G = B^T S^T Y_l E^T / rho (B X as scratch)
        st = f64 ? Impl<double>::sb_data_term(c, c->stream) : Impl<float>::sb_data_term(c, c->stream);
        if (st != FUSE_OK) return st;
    }
    st = run_iterations(c, iters, cold);
    if (st != FUSE_OK) return st;
    if (c->monitor && iters > 0) c->mon_epoch = c->epoch;
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
    ++c->epoch;
    if (c->dtype == FUSE_F64) st = Impl<double>::weights<double>(c, G);
    else if (c->wdtype == FUSE_BF16) st = Impl<float>::weights<__nv_bfloat16>(c, G);
    else st = Impl<float>::weights<float>(c, G);
    if (st == FUSE_OK) c->have_weights = true;
    return st;
}

void grad_free(GradWork* g);

// Reallocates the latent state for half-window mode `h` and storage format `f`; clears the
// ADMM state (the next solve starts from zero) and the captured iteration graph.
fuse_status realloc_state(fuse_ctx* c, int h, int f) {
    const size_t nWs = h ? (size_t)c->nW / 2 : (size_t)c->nW;
    const size_t bytes = nWs * c->nP * c->Ls * c->n * (f ? 2 : c->esz);
    for (auto& p : c->allocs)
        if (p == c->Sig) { CK(c, cudaStreamSynchronize(c->stream)); cudaFree(p); p = nullptr; }
    c->Sig = nullptr;
    fuse_status s2 = dalloc(c, &c->Sig, bytes);
    if (s2 != FUSE_OK) return s2;
    c->sig_bytes = bytes;
    c->half = h;
    c->sfmt = f;
    latent_tma_shape(c);
    ++c->epoch;
    c->have_state = false;
    c->have_x = false;
    drop_graphs(c);
    return FUSE_OK;
}

void release(fuse_ctx* c) {
    grad_free(c->gw);
    c->gw = nullptr;
    drop_graphs(c);
    for (auto& e : c->ev) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (void* p : c->allocs)
        if (p) cudaFree(p);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->side.destroy();
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

// Tables and launch shape of the column pass of the variant with S B in the X system, in FP64 on
// the host (see fft_cols_alias_kernel):
//   b^(u,v) = sum_{a,b} blur(a,b) exp(-2 pi i (u (a - bh/2)/H + v (b - bw/2)/W)),
//   g = 1 + |P| (2|W| - 2 (Cu Cv - 1)),  p = b^/g,  q = 1/(g H W),
//   kappa(class) = beta / ((1 + beta sum_class |b^|^2/g) H W),  beta = eps / (rho d^2).
fuse_status sb_prepare(fuse_ctx* c) {
    const int H = c->H, W = c->W, d = c->d, h = H / d, w = W / d;
    // shape: m base columns (m d columns) per block, 2H+1 complex values per column in shared memory
    const size_t csz = 2 * c->esz;
    int m = d >= 8 ? 1 : 8 / d;
    if (m > w) m = w;
    while (m > 1 && (size_t)m * d * (2 * H + 1) * csz > kMaxSmem) m /= 2;
    // fewer base columns per block until the pass has about four blocks per SM
    while (m > 1 && (long long)((w + m - 1) / m) * c->npair < 4 * c->nsm) m /= 2;
    if ((size_t)m * d * (2 * H + 1) * csz > kMaxSmem || m * d > 256)
        return fail(c, FUSE_EUNSUPPORTED, "the alias-class column pass does not fit shared memory");
    int tpc = H / 4 < 1 ? 1 : H / 4;
    while (tpc > 1 && m * d * tpc > 256) tpc /= 2;
    if (!c->sbq) {
        const double tp = 2.0 * M_PI;
        const int rh = c->bh / 2, rw = c->bw / 2;
        std::vector<double> q(c->n), pf(2 * c->n), kap((size_t)h * w, 0.0), b2g(c->n);
        std::vector<double> Cu(H), Cv(W);
        for (int u = 0; u < H; ++u) { double t = 0; for (int k = -c->S; k <= c->S; ++k) t += std::cos(tp * u * k / H); Cu[u] = t; }
        for (int v = 0; v < W; ++v) { double t = 0; for (int k = -c->S; k <= c->S; ++k) t += std::cos(tp * v * k / W); Cv[v] = t; }
        // row sums over b first: gr + i gi = sum_b blur(a,b) exp(-2 pi i v (b - bw/2)/W)
        std::vector<double> gr((size_t)c->bh * W), gi((size_t)c->bh * W);
        for (int a = 0; a < c->bh; ++a)
            for (int v = 0; v < W; ++v) {
                double sr = 0, si = 0;
                for (int b = 0; b < c->bw; ++b) {
                    const double ang = -tp * (double)v * (double)(b - rw) / W;
                    sr += c->htapsT[(size_t)a * c->bw + b] * std::cos(ang);
                    si += c->htapsT[(size_t)a * c->bw + b] * std::sin(ang);
                }
                gr[(size_t)a * W + v] = sr;
                gi[(size_t)a * W + v] = si;
            }
        for (int u = 0; u < H; ++u)
            for (int v = 0; v < W; ++v) {
                double br = 0, bi = 0;
                for (int a = 0; a < c->bh; ++a) {
                    const double ang = -tp * (double)u * (double)(a - rh) / H;
                    const double er = std::cos(ang), ei = std::sin(ang);
                    const double xr = gr[(size_t)a * W + v], xi = gi[(size_t)a * W + v];
                    br += er * xr - ei * xi;
                    bi += er * xi + ei * xr;
                }
                const double g = 1.0 + (double)c->nP * (2.0 * c->nW - 2.0 * (Cu[u] * Cv[v] - 1.0));
                const size_t i = (size_t)u * W + v;
                q[i] = 1.0 / (g * (double)H * (double)W);
                pf[2 * i] = br / g;
                pf[2 * i + 1] = bi / g;
                b2g[i] = (br * br + bi * bi) / g;
                kap[(size_t)(u % h) * w + (v % w)] += b2g[i];
            }
        const double beta = c->eet_eps / (c->rho * (double)d * (double)d);
        for (double& t : kap) t = beta / ((1.0 + beta * t) * (double)H * (double)W);
        fuse_status st;
        if ((st = upload_any(c, &c->sbq, q)) != FUSE_OK) return st;
        if ((st = upload_any(c, &c->sbp, pf)) != FUSE_OK) return st;
        if ((st = upload_any(c, &c->sbk, kap)) != FUSE_OK) return st;
    }
    c->fa_m = m;
    c->fa_tpc = tpc;
    c->fa_smem = (size_t)m * d * (2 * H + 1) * csz;
    return FUSE_OK;
}


}  // namespace

// ---------------------------------------------------------------------------------------
// batches of independent problems of uneven sizes: one launch per ADMM phase
// ---------------------------------------------------------------------------------------

struct fuse_batch {
    std::vector<fuse_ctx*> ctx;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    SideBranch side;
    int device = 0;
    fuse_dtype dtype = FUSE_F32, wdtype = FUSE_F32;
    int K = 0, S = 0, Ls = 0, bh = 1, bw = 1, half = 1, sfmt = 0;
    bool same_taps = false;     // every problem has the same blur taps
    // launch shapes shared by all problems
    int lat_target = 256, lat_stages = 6, lat_ncons = 0, lat_bpb = 2;
    size_t lat_smem = 0, st_smem = 0, fr_smem = 0, fc_smem = 0, px_smem = 0;
    int fr_rpb = 4, fc_cw = 8;
    // device tables: [args of every problem] and segments per kernel
    void* d_lat = nullptr; Segment* d_lat_seg = nullptr; int lat_nseg = 0, lat_blocks = 0;
    void* d_st1 = nullptr; void* d_st0 = nullptr; Segment* d_st_seg = nullptr; int st_nseg = 0, st_blocks = 0;
    // separable B X: blocks of stencil_sep_bands bands (band groups in z)
    Segment* d_sep0_seg = nullptr; int sep0_nseg = 0, sep0_blocks = 0;
    void* d_fft = nullptr; Segment* d_fr_seg = nullptr; Segment* d_fc_seg = nullptr;
    int fr_nseg = 0, fr_blocks = 0, fc_nseg = 0, fc_blocks = 0;
    void* d_px = nullptr; Segment* d_px_seg = nullptr; int px_nseg = 0, px_blocks = 0;
    std::vector<void*> allocs;
    bool profile = false, use_graph = true;
    LoopCache loops;
    std::vector<Event2> ev;
    size_t ev_used = 0;
    double latent_ms = 0.0;
    long long launches_all = 0, launches_latent = 0;
    fuse_status sticky = FUSE_OK;
    std::string err;
};

namespace {

fuse_status bfail(fuse_batch* b, fuse_status s, const std::string& msg) {
    if (b) {
        if (b->sticky == FUSE_OK) b->sticky = s;
        b->err = msg;
    }
    return s;
}

#define BCK(b, expr)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            char m_[512];                                                                     \
            snprintf(m_, sizeof m_, "%s: %s", #expr, cudaGetErrorString(e_));                 \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? FUSE_ENOMEM : FUSE_ECUDA, m_); \
        }                                                                                     \
    } while (0)

template <typename V>
fuse_status bupload(fuse_batch* b, void** dst, const std::vector<V>& v) {
    cudaError_t e = cudaMalloc(dst, v.size() * sizeof(V) + 16);
    if (e != cudaSuccess) { *dst = nullptr; cudaGetLastError(); return bfail(b, FUSE_ENOMEM, "cudaMalloc (batch tables)"); }
    b->allocs.push_back(*dst);
    BCK(b, cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
    return FUSE_OK;
}

// Appends the segments of one problem's (gx, gy, gz) grid starting at block `*next`.
void add_segment(std::vector<Segment>& seg, int prob, int gx, int gy, int gz, int z0, int* next) {
    if (gx <= 0 || gy <= 0 || gz <= 0) return;
    seg.push_back(Segment{prob, *next, gx, gy, gz, z0});
    *next += gx * gy * gz;
}

template <typename T, typename WT>
struct BatchImpl {
    static constexpr int VEC = 32 / sizeof(T);          // pixels per thread of the latent pass

    static fuse_status build(fuse_batch* b) {
        const int n = (int)b->ctx.size();
        const size_t esz = sizeof(T), csz = 2 * sizeof(T);
        const int side = 2 * b->S + 1;
        const int rows = b->half ? b->S + 1 : side;
        // latent: per-problem Ty, common consumer count and ring depth
        std::vector<LatentArgs<T, WT>> la(n);
        std::vector<int> Ty(n);
        b->lat_ncons = 32;
        for (int i = 0; i < n; ++i) {
            fuse_ctx* c = b->ctx[i];
            if (c->W % VEC) return bfail(b, FUSE_EUNSUPPORTED, "batched problems need W a multiple of 32 bytes of pixels");
            const int tpr = c->W / VEC;
            int ty = b->lat_target / tpr;
            ty = ty < 1 ? 1 : (ty > c->H ? c->H : ty);
            while (ty > 1 && ((tpr * ty + 31) / 32) * 32 + 32 > 288) --ty;
            const int nc = ((tpr * ty + 31) / 32) * 32;
            if (nc + 32 > 288) return bfail(b, FUSE_EUNSUPPORTED, "image too wide for the batched latent pass");
            Ty[i] = ty;
            if (nc > b->lat_ncons) b->lat_ncons = nc;
        }
        b->lat_smem = 0;
        for (int i = 0; i < n; ++i) {
            fuse_ctx* c = b->ctx[i];
            la[i] = Impl<T>::template lat_args<WT>(c, Ty[i], b->lat_ncons, b->lat_stages, b->lat_bpb);
            const size_t ssz = b->sfmt ? 2 : esz;
            const size_t sm = (size_t)b->lat_stages * Ty[i] * c->W * ssz + 5 * (size_t)Ty[i] * c->W * esz +
                              2 * (size_t)b->lat_stages * 8;
            if (sm > b->lat_smem) b->lat_smem = sm;
        }
        if (b->lat_smem > (size_t)kMaxSmem) return bfail(b, FUSE_EUNSUPPORTED, "batched latent ring exceeds shared memory");
        std::vector<Segment> seg;
        int next = 0;
        const int groups = (b->Ls + b->lat_bpb - 1) / b->lat_bpb;
        for (int i = 0; i < n; ++i)          // heavy block rows (tau1 != 0) of every problem first
            add_segment(seg, i, (b->ctx[i]->H + Ty[i] - 1) / Ty[i], groups, rows - 1, 0, &next);
        for (int i = 0; i < n; ++i)          // then the lighter tau1 = 0 rows
            add_segment(seg, i, (b->ctx[i]->H + Ty[i] - 1) / Ty[i], groups, 1, rows - 1, &next);
        b->lat_nseg = (int)seg.size();
        b->lat_blocks = next;
        fuse_status st;
        if ((st = bupload(b, &b->d_lat, la)) != FUSE_OK) return st;
        if ((st = bupload(b, (void**)&b->d_lat_seg, seg)) != FUSE_OK) return st;

        // stencils (same blur for all problems)
        std::vector<StencilArgs<T>> s1(n), s0(n);
        seg.clear();
        next = 0;
        for (int i = 0; i < n; ++i) {
            fuse_ctx* c = b->ctx[i];
            s1[i] = Impl<T>::st_args(c, c->U1, c->C, c->tapsT);
            s0[i] = Impl<T>::st_args(c, c->X, c->BX, c->tapsB);
            add_segment(seg, i, (c->W + ST_TX - 1) / ST_TX, (c->H + ST_TY - 1) / ST_TY, b->Ls, 0, &next);
        }
        b->st_smem = b->ctx[0]->st_smem;
        b->st_nseg = (int)seg.size();
        b->st_blocks = next;
        if ((st = bupload(b, &b->d_st1, s1)) != FUSE_OK) return st;
        if ((st = bupload(b, &b->d_st0, s0)) != FUSE_OK) return st;
        if ((st = bupload(b, (void**)&b->d_st_seg, seg)) != FUSE_OK) return st;
        {
            constexpr int NB = stencil_sep_bands<T, 0>();
            std::vector<Segment> sg;
            int nx = 0;
            for (int i = 0; i < n; ++i) {
                fuse_ctx* c = b->ctx[i];
                add_segment(sg, i, (c->W + ST_TX - 1) / ST_TX, (c->H + ST_TY - 1) / ST_TY, (b->Ls + NB - 1) / NB, 0,
                            &nx);
            }
            b->sep0_nseg = (int)sg.size();
            b->sep0_blocks = nx;
            if ((st = bupload(b, (void**)&b->d_sep0_seg, sg)) != FUSE_OK) return st;
        }

        // FFT passes: 256 threads; each problem in its context's form (register-resident: 8 rows
        // or 8 columns per block, one warp each; Stockham: rpb rows, tpr = 256 / rpb, or CW
        // columns per block)
        std::vector<FFTArgs<T>> fa(n);
        std::vector<Segment> sr, sc;
        int nr = 0, ncl = 0;
        b->fr_smem = b->fc_smem = 0;
        for (int i = 0; i < n; ++i) {
            fuse_ctx* c = b->ctx[i];
            const int rpb = b->fr_rpb;
            fa[i] = Impl<T>::fft_args(c, rpb, b->fc_cw);
            if (fa[i].fT) {
                add_segment(sr, i, (c->H + 7) / 8, c->npair, 1, 0, &nr);
                add_segment(sc, i, (c->W + kWfftCols - 1) / kWfftCols, c->npair, 1, 0, &ncl);
                const size_t cc = wfft_cols_smem<T>(c->H);
                if (cc > b->fc_smem) b->fc_smem = cc;
                continue;
            }
            add_segment(sr, i, (c->H + rpb - 1) / rpb, c->npair, 1, 0, &nr);
            add_segment(sc, i, (c->W + b->fc_cw - 1) / b->fc_cw, c->npair, 1, 0, &ncl);
            const size_t r = 2 * (size_t)rpb * c->W * csz;
            const size_t cc = (size_t)b->fc_cw * (2 * c->H + 1) * csz;
            if (r > b->fr_smem) b->fr_smem = r;
            if (cc > b->fc_smem) b->fc_smem = cc;
        }
        if (b->fr_smem > (size_t)kMaxSmem || b->fc_smem > (size_t)kMaxSmem)
            return bfail(b, FUSE_EUNSUPPORTED, "image too large for the batched FFT");
        b->fr_nseg = (int)sr.size(); b->fr_blocks = nr;
        b->fc_nseg = (int)sc.size(); b->fc_blocks = ncl;
        if ((st = bupload(b, &b->d_fft, fa)) != FUSE_OK) return st;
        if ((st = bupload(b, (void**)&b->d_fr_seg, sr)) != FUSE_OK) return st;
        if ((st = bupload(b, (void**)&b->d_fc_seg, sc)) != FUSE_OK) return st;

        // pixel updates
        std::vector<PixelArgs<T>> pa(n);
        seg.clear();
        next = 0;
        for (int i = 0; i < n; ++i) {
            fuse_ctx* c = b->ctx[i];
            pa[i] = Impl<T>::px_args(c);
            add_segment(seg, i, (int)((c->n + 127) / 128), 1, 1, 0, &next);
        }
        b->px_smem = 2 * (size_t)b->Ls * b->Ls * esz;
        b->px_nseg = (int)seg.size();
        b->px_blocks = next;
        if ((st = bupload(b, &b->d_px, pa)) != FUSE_OK) return st;
        if ((st = bupload(b, (void**)&b->d_px_seg, seg)) != FUSE_OK) return st;

        // attributes
        BCK(b, (latent_batch_set_smem<T, WT>(b->K, kMaxSmem)));
        BCK(b, stencil_batch_set_smem<T>(b->bh, kMaxSmem));
        BCK(b, wfft_set_smem<T>(kMaxSmem));
        return FUSE_OK;
    }

    // One batched ADMM iteration: 7 launches cover every problem.  zero_in: the latent state of
    // every problem is zero on entry (first iteration of the solve) and is not read.
    // side, join_prev: as for a single problem (B X and the pixel pass beside the latent pass in
    // captured loops).
    static fuse_status iterate(fuse_batch* b, cudaStream_t s, bool timed, bool zero_in = false, bool side = false,
                               bool join_prev = false) {
        if (side && join_prev) BCK(b, cudaStreamWaitEvent(s, b->side.join, 0));
        // square blurs shared by every problem: taps in the argument space (from problem 0)
        const fuse_ctx* c0 = b->ctx[0];
        const bool sq = b->bh == b->bw && b->same_taps;
        const bool sep = sq && c0->sep_blur && !c0->hsepT.empty();
        stencil_batch_launch<T, 1>((const StencilArgs<T>*)b->d_st1, b->d_st_seg, b->st_nseg, b->bh,
                                   sep ? c0->hsepT.data() : nullptr, sq ? c0->htapsT.data() : nullptr,
                                   (unsigned)b->st_blocks, b->st_smem, s, b->Ls);
        const FFTArgs<T>* fa = (const FFTArgs<T>*)b->d_fft;
        fft_batch_launch<T>(fa, b->d_fr_seg, b->fr_nseg, 0, (unsigned)b->fr_blocks, b->fr_smem, s);
        fft_batch_launch<T>(fa, b->d_fc_seg, b->fc_nseg, 1, (unsigned)b->fc_blocks, b->fc_smem, s);
        fft_batch_launch<T>(fa, b->d_fr_seg, b->fr_nseg, 2, (unsigned)b->fr_blocks, b->fr_smem, s);
        cudaStream_t sp = s;
        if (side) {
            BCK(b, cudaEventRecord(b->side.fork, s));
            BCK(b, cudaStreamWaitEvent(b->side.s, b->side.fork, 0));
            sp = b->side.s;
        }
        stencil_batch_launch<T, 0>((const StencilArgs<T>*)b->d_st0, sep ? b->d_sep0_seg : b->d_st_seg,
                                   sep ? b->sep0_nseg : b->st_nseg, b->bh, sep ? c0->hsepB.data() : nullptr,
                                   sq ? c0->htapsB.data() : nullptr,
                                   (unsigned)(sep ? b->sep0_blocks : b->st_blocks), b->st_smem, sp, b->Ls);
        pixel_batch_launch<T>((const PixelArgs<T>*)b->d_px, b->d_px_seg, b->px_nseg, b->Ls, (unsigned)b->px_blocks,
                              b->px_smem, sp);
        if (side) BCK(b, cudaEventRecord(b->side.join, b->side.s));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            if (b->ev_used == b->ev.size()) {
                Event2 e{};
                BCK(b, cudaEventCreate(&e.a));
                BCK(b, cudaEventCreate(&e.b));
                b->ev.push_back(e);
            }
            e0 = b->ev[b->ev_used].a;
            e1 = b->ev[b->ev_used].b;
            b->ev_used++;
            BCK(b, cudaEventRecord(e0, s));
        }
        latent_tma_batch_launch<T, WT>((const LatentArgs<T, WT>*)b->d_lat, b->d_lat_seg, b->lat_nseg, zero_in ? 1 : 0,
                                       b->K, b->sfmt != 0, (unsigned)b->lat_blocks, (unsigned)(b->lat_ncons + 32),
                                       b->lat_smem, s);
        if (timed) BCK(b, cudaEventRecord(e1, s));
        BCK(b, cudaGetLastError());
        return FUSE_OK;
    }
};

fuse_status batch_build(fuse_batch* b) {
    if (b->dtype == FUSE_F64) return BatchImpl<double, double>::build(b);
    if (b->wdtype == FUSE_BF16) return BatchImpl<float, __nv_bfloat16>::build(b);
    return BatchImpl<float, float>::build(b);
}

fuse_status batch_iterate(fuse_batch* b, cudaStream_t s, bool timed, bool zero_in = false, bool side = false,
                          bool join_prev = false) {
    if (b->dtype == FUSE_F64) return BatchImpl<double, double>::iterate(b, s, timed, zero_in, side, join_prev);
    if (b->wdtype == FUSE_BF16)
        return BatchImpl<float, __nv_bfloat16>::iterate(b, s, timed, zero_in, side, join_prev);
    return BatchImpl<float, float>::iterate(b, s, timed, zero_in, side, join_prev);
}

void batch_release(fuse_batch* b) {
    b->loops.clear();
    for (auto& e : b->ev) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    b->ev.clear();
    for (void* p : b->allocs) if (p) cudaFree(p);
    b->allocs.clear();
}

// Sets the batch's latent launch shape (consumer threads, ring slots, bands per block) and rebuilds
// its launch tables once; a shape that does not fit leaves the previous one in place (FUSE_EINVAL).
fuse_status batch_set_shape(fuse_batch* b, int threads, int stages, int bands) {
    if (threads < 32 || threads > 256 || stages < 2 || stages > 32 || bands < 1 || bands > 64)
        return bfail(b, FUSE_EINVAL, "latent launch option out of range");
    const int old_t = b->lat_target, old_d = b->lat_stages, old_b = b->lat_bpb;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    b->lat_target = threads;
    b->lat_stages = stages;
    b->lat_bpb = bands;
    if (batch_build(b) == FUSE_OK) return FUSE_OK;
    b->sticky = FUSE_OK;
    b->lat_target = old_t; b->lat_stages = old_d; b->lat_bpb = old_b;
    batch_release(b);
    if (batch_build(b) != FUSE_OK) return bfail(b, FUSE_ECUDA, "cannot rebuild the batch tables");
    return bfail(b, FUSE_EINVAL, "latent launch shape does not fit the batch");
}

// Batched counterpart of launch_loop: `len` batched iterations replayed from one graph.
fuse_status batch_launch_loop(fuse_batch* b, int len, bool cold) {
    LoopGraph* lg = b->loops.find(len, cold);
    if (!lg) {
        BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        fuse_status st = FUSE_OK;
        int forked = 0;
        for (int t = 0; t < len && st == FUSE_OK; ++t, ++forked)
            st = batch_iterate(b, b->cap_stream, false, cold && t == 0, true, t > 0);
        // the side branch of the last iteration joins the loop's stream before the capture ends
        if (forked && cudaStreamWaitEvent(b->cap_stream, b->side.join, 0) != cudaSuccess && st == FUSE_OK)
            st = bfail(b, FUSE_ECUDA, "cudaStreamWaitEvent");
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != FUSE_OK) { if (g) cudaGraphDestroy(g); return st; }
        BCK(b, e);
        lg = b->loops.victim();
        if (lg->exec) cudaGraphExecDestroy(lg->exec);
        *lg = LoopGraph{};
        e = cudaGraphInstantiate(&lg->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { lg->exec = nullptr; BCK(b, e); }
        lg->len = len;
        lg->cold = cold;
        lg->launches = 7LL * len;
        lg->used = ++b->loops.tick;
    }
    BCK(b, cudaGraphLaunch(lg->exec, b->stream));
    b->launches_all += lg->launches;
    b->launches_latent += len;
    return FUSE_OK;
}

// `iters` batched iterations (whole loop in graphs of up to kGraphIters iterations, or direct
// launches when profiling or with graphs off); cold as in run_iterations.
fuse_status batch_run(fuse_batch* b, int iters, bool cold = false) {
    if (iters <= 0) return FUSE_OK;
    if (b->profile || !b->use_graph) {
        for (int t = 0; t < iters; ++t) {
            fuse_status st = batch_iterate(b, b->stream, b->profile, cold && t == 0);
            if (st != FUSE_OK) return st;
            b->launches_all += 7;
            b->launches_latent += 1;
        }
        return FUSE_OK;
    }
    for (int done = 0; done < iters;) {
        const int len = std::min(iters - done, kGraphIters);
        fuse_status st = batch_launch_loop(b, len, cold && done == 0);
        if (st != FUSE_OK) return st;
        done += len;
    }
    return FUSE_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------------------

#include "grad_impl.cuh"

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
    // the launch shapes for this device's SM count
    int dev = 0, nsm = kDefaultSMs;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
        cudaGetLastError();
        return FUSE_ECUDA;
    }
    if ((st = check_geometry(nullptr, g, K, S, ratio, dtype, wdtype, bh, bw, &sh, &pH, &pW, nsm)) != FUSE_OK) return st;

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
    c->nsm = nsm;

    auto bail = [&](fuse_status s) { release(c); delete c; return s; };
    if (cudaGetDevice(&c->device) != cudaSuccess) { cudaGetLastError(); return bail(FUSE_ECUDA); }
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess || !c->side.create()) {
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
    {
        // E E^T = eps I test for the variant with S B in the X system
        double tr = 0.0;
        for (int i = 0; i < Ls; ++i) tr += M1[(size_t)i * Ls + i] - rho;
        c->eet_eps = tr / Ls;
        double dev = 0.0;
        for (int i = 0; i < Ls; ++i)
            for (int j = 0; j < Ls; ++j)
                dev = std::max(dev, std::fabs(M1[(size_t)i * Ls + j] - (i == j ? rho + c->eet_eps : 0.0)));
        c->eet_dev = c->eet_eps > 0 ? dev / c->eet_eps : INFINITY;
    }
    {
        // conditioning (before inversion): E E^T + rho I and F^{-1} = I + lambda1/rho E R R^T E^T;
        // A = I + B^T B + sum D^T D is diagonal in the DFT basis with eigenvalues 1/(HW f)
        double lo, hi;
        sym_eig_range(M1, Ls, &lo, &hi);
        c->cond[1] = hi / lo;
        sym_eig_range(Fm, Ls, &lo, &hi);
        c->cond[2] = hi / lo;
        double fmin = fh[0], fmax = fh[0];
        for (double v : fh) { fmin = std::min(fmin, v); fmax = std::max(fmax, v); }
        c->cond[0] = fmax / fmin;
    }
    if (!invert(M1, Ls) || !invert(Fm, Ls)) return bail(FUSE_EINVAL);
    c->htapsT = tT;
    c->htapsB = tB;
    if (bh == bw) {
        c->hsepT = separable_factors(tT, bh);
        c->hsepB = separable_factors(tB, bh);
    }
    c->hM1 = M1;
    c->hF = Fm;
    c->hER = ER;
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
    if (wfft_length_ok(H) && wfft_length_ok(W)) {
        // f in the register-resident form's spectrum order: fT[q][r] = f(u(r), v(q)) for row
        // position r and column position q, u(r) = r / 32 + (H / 32) rev5(r mod 32), v likewise
        auto freq = [](int pos, int P) {
            int r = 0;
            for (int b = 0; b < 5; ++b) r |= ((pos >> b) & 1) << (4 - b);
            return pos / 32 + P * r;
        };
        std::vector<double> ft(c->n);
        for (int q = 0; q < W; ++q) {
            const int v = freq(q, W / 32);
            for (int r = 0; r < H; ++r) ft[(size_t)q * H + r] = fh[(size_t)freq(r, H / 32) * W + v];
        }
        if ((st = upload_any(c, &c->fT, ft)) != FUSE_OK) return bail(st);
        c->fft_impl = 1;
    }
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
    ++c->epoch;
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

fuse_status fuse_residuals(fuse_ctx* c, double out[2]) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!out) return fail(c, FUSE_EINVAL, "NULL argument");
    if (!c->monitor || !c->mon_part || c->mon_epoch != c->epoch)
        return fail(c, FUSE_ESTATE, "no monitored iteration since the last change of inputs or state");
    const size_t np = c->mon_lat_cap + 2 * kMonBlocks;
    std::vector<double> h(np);
    CK(c, cudaMemcpyAsync(h.data(), c->mon_part, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    double lat = 0.0, pix = 0.0, dual = 0.0;
    for (size_t b = 0; b < c->mon_lat; ++b) lat += h[b];
    for (int b = 0; b < kMonBlocks; ++b) {
        pix += h[c->mon_lat_cap + b];
        dual += h[c->mon_lat_cap + kMonBlocks + b];
    }
    // half-window mode: the -tau offsets' latent variables are images of the kept ones under an
    // orthogonal map, so their squared norms are equal
    out[0] = std::sqrt(pix + (c->half ? 2.0 : 1.0) * lat);
    out[1] = c->rho * std::sqrt(dual);
    if (!std::isfinite(out[0]) || !std::isfinite(out[1])) return fail(c, FUSE_ENONFINITE, "residual is not finite");
    return FUSE_OK;
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
    ++c->epoch;
    return FUSE_OK;
}

fuse_status fuse_set_option(fuse_ctx* c, int option, long long value) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    switch (option) {
        case FUSE_OPT_PROFILE: c->profile = value != 0; return FUSE_OK;
        case FUSE_OPT_GRAPH: c->use_graph = value != 0; return FUSE_OK;
        case FUSE_OPT_GRAD_SEGMENT:
            if (value < 0 || value > (1 << 30)) return fail(c, FUSE_EINVAL, "iterations per segment must be >= 0");
            c->grad_seg = (int)value;
            return FUSE_OK;
        case FUSE_OPT_GRAD_WEIGHTS: c->grad_weights = value != 0; return FUSE_OK;
        case FUSE_OPT_LATENT_BANDS:
            if (value < 1 || value > 64) return fail(c, FUSE_EINVAL, "bands per latent block must be in [1, 64]");
            c->lat_bpb = (int)value;
            drop_graphs(c);
            return FUSE_OK;
        case FUSE_OPT_LATENT_IMPL:
        case FUSE_OPT_LATENT_THREADS:
        case FUSE_OPT_LATENT_STAGES: {
            if (option == FUSE_OPT_LATENT_IMPL && !value && c->sfmt)
                return fail(c, FUSE_EUNSUPPORTED, "the fixed-point state needs the bulk-copy latent pass");
            const int old_impl = c->lat_impl, old_t = c->lat_target, old_d = c->lat_stages;
            if (option == FUSE_OPT_LATENT_IMPL) c->lat_impl = value ? 1 : 0;
            if (option == FUSE_OPT_LATENT_THREADS) c->lat_target = (int)value;
            if (option == FUSE_OPT_LATENT_STAGES) c->lat_stages = (int)value;
            if (c->lat_target < 32 || c->lat_target > 256 || c->lat_stages < 2 || c->lat_stages > 32 ||
                (c->lat_impl == 1 && !latent_tma_shape(c))) {
                c->lat_impl = old_impl; c->lat_target = old_t; c->lat_stages = old_d;
                latent_tma_shape(c);
                return fail(c, FUSE_EINVAL, "latent launch option out of range");
            }
            drop_graphs(c);
            return FUSE_OK;
        }
        case FUSE_OPT_FFT_ROWS: {
            const int rpb = (int)value;
            const size_t csz = 2 * c->esz;
            if (rpb < 1 || rpb > 8 || (rpb & (rpb - 1)) || 2 * (size_t)rpb * c->W * csz > (size_t)kMaxSmem)
                return fail(c, FUSE_EINVAL, "FFT rows per block must be 1, 2, 4 or 8 and fit shared memory");
            c->fr_rpb = rpb;
            c->fr_tpr = 256 / rpb;
            c->fr_smem = 2 * (size_t)rpb * c->W * csz;
            drop_graphs(c);
            return FUSE_OK;
        }
        case FUSE_OPT_FFT_COLS: {
            const int cw = (int)value;
            const size_t csz = 2 * c->esz;
            if (cw < 1 || cw > 32 || (cw & (cw - 1)) || (size_t)cw * (2 * c->H + 1) * csz > (size_t)kMaxSmem)
                return fail(c, FUSE_EINVAL, "FFT columns per block must be a power of 2 <= 32 and fit shared memory");
            c->fc_cw = cw;
            c->fc_tpc = 256 / cw;
            c->fc_smem = (size_t)cw * (2 * c->H + 1) * csz;
            drop_graphs(c);
            return FUSE_OK;
        }
        case FUSE_OPT_HALF_WINDOW: {
            const int h = value ? 1 : 0;
            if (h == c->half) return FUSE_OK;
            return realloc_state(c, h, c->sfmt);
        }
        case FUSE_OPT_STATE_FORMAT: {
            const int f = value ? 1 : 0;
            if (f == c->sfmt) return FUSE_OK;
            if (f == 1) {
                if (c->dtype != FUSE_F32) return fail(c, FUSE_EUNSUPPORTED, "fixed-point state needs an F32 context");
                const int old_impl = c->lat_impl;
                c->sfmt = 1;
                c->lat_impl = 1;
                if (!latent_tma_shape(c)) {
                    c->sfmt = 0;
                    c->lat_impl = old_impl;
                    latent_tma_shape(c);
                    return fail(c, FUSE_EUNSUPPORTED, "fixed-point state needs the bulk-copy latent pass (W % 8 == 0)");
                }
                c->sfmt = 0;
            }
            return realloc_state(c, c->half, f);
        }
        case FUSE_OPT_X_UPDATE: {
            if (value != 0 && value != 1) return fail(c, FUSE_EINVAL, "X update is 0 or 1");
            if (value == c->xmode) return FUSE_OK;
            if (value == 1) {
                if (c->mask) return fail(c, FUSE_EUNSUPPORTED, "the S B-in-X update needs the regular lattice");
                if (!(c->eet_dev <= 1e-6))
                    return fail(c, FUSE_EUNSUPPORTED, "the S B-in-X update needs E E^T = eps I");
                if ((st = sb_prepare(c)) != FUSE_OK) return st;
            }
            c->xmode = (int)value;
            ++c->epoch;
            c->have_state = false;
            c->have_x = false;
            drop_graphs(c);
            return FUSE_OK;
        }
        case FUSE_OPT_SEPARABLE_BLUR:
            if (value != 0 && value != 1) return fail(c, FUSE_EINVAL, "separable blur is 0 or 1");
            c->sep_blur = (int)value;
            drop_graphs(c);
            return FUSE_OK;
        case FUSE_OPT_FFT_IMPL:
            if (value != 0 && value != 1) return fail(c, FUSE_EINVAL, "FFT form is 0 or 1");
            if (value == 1 && !c->fT)
                return fail(c, FUSE_EUNSUPPORTED, "the register-resident FFT needs H and W = 32 P, P in "
                                                  "{1, 2, 3, 4, 5, 6, 8, 10, 12, 16}");
            c->fft_impl = (int)value;
            drop_graphs(c);
            return FUSE_OK;
        case FUSE_OPT_RESIDUALS: {
            if (value != 0 && value != 1) return fail(c, FUSE_EINVAL, "residual monitor is 0 or 1");
            if (value == 1 && (c->xmode != 0 || c->sfmt != 0 || c->lat_impl != 1))
                return fail(c, FUSE_EUNSUPPORTED, "the residual monitor needs the bulk-copy latent pass, the state "
                                                  "in the iterate type and the paper's splitting");
            if (value == 1 && !c->mon_part) {
                const size_t img = c->n * c->Ls * c->esz;
                void** imgs[] = {&c->mL1, &c->mU1, &c->mL2, &c->mU2};
                for (void** q : imgs)
                    if ((st = dalloc(c, q, img)) != FUSE_OK) return st;
                if ((st = dalloc(c, &c->mPo, c->plane_bytes)) != FUSE_OK) return st;
                if ((st = dalloc(c, &c->mPm, c->plane_bytes)) != FUSE_OK) return st;
                // latent blocks are at most H * L_s * (2S+1) (one row and one band per block)
                c->mon_lat_cap = (size_t)c->H * c->Ls * (2 * c->S + 1);
                if ((st = dalloc(c, (void**)&c->mon_part, (c->mon_lat_cap + 2 * kMonBlocks) * sizeof(double))) != FUSE_OK)
                    return st;
                if (!set_monitor_smem(c)) return fail(c, FUSE_ECUDA, "cudaFuncSetAttribute (monitoring latent pass)");
            }
            c->monitor = (int)value;
            return FUSE_OK;
        }
        case FUSE_OPT_WAIT_LIMIT:
            if (value < 1) return fail(c, FUSE_EINVAL, "wait limit must be positive");
            c->wait_limit = (unsigned)value;
            drop_graphs(c);
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

// Device time of `iters` iterations (direct launches) of the current configuration, in ms.
static fuse_status time_iterations(fuse_ctx* c, int iters, double* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(c, cudaEventCreate(&a));
    CK(c, cudaEventCreate(&b));
    const bool g = c->use_graph, pr = c->profile;
    const int mon = c->monitor;
    c->use_graph = false;
    c->profile = false;
    c->monitor = 0;
    fuse_status st = run_iterations(c, 1);                 // warm-up
    if (st == FUSE_OK) {
        cudaEventRecord(a, c->stream);
        st = run_iterations(c, iters);
        cudaEventRecord(b, c->stream);
    }
    c->use_graph = g;
    c->profile = pr;
    c->monitor = mon;
    float t = 0.f;
    if (st == FUSE_OK && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess)
        *ms = t;
    else if (st == FUSE_OK)
        st = fail(c, FUSE_ECUDA, "autotune timing failed");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

fuse_status fuse_autotune(fuse_ctx* c, const void* Yl, const void* Yh, int iters) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!Yl || !Yh || iters < 1) return fail(c, FUSE_EINVAL, "autotune needs inputs and iters >= 1");
    if (!c->have_weights) return FUSE_ESTATE;
    // inputs and a zero state (the timed iterations run on it; the next solve starts over)
    st = solve_impl(c, Yl, Yh, 0, 0, nullptr, nullptr);
    if (st != FUSE_OK) return st;
    double best = 1e30, t = 0;
    // 1. latent pass: ring shape and bands per block
    if (c->lat_impl == 1) {
        const int bt = c->lat_target, bs = c->lat_stages, bb = c->lat_bpb;
        int best_t = bt, best_s = bs, best_b = bb;
        const int threads[] = {128, 192, 256}, stages[] = {4, 6, 8, 12, 16, 24}, bands[] = {1, 2};
        for (int th : threads)
            for (int sg : stages)
                for (int bd : bands) {
                    c->lat_target = th; c->lat_stages = sg; c->lat_bpb = bd;
                    if (!latent_tma_shape(c)) continue;
                    if ((st = time_iterations(c, iters, &t)) != FUSE_OK) return st;
                    if (t < best) { best = t; best_t = th; best_s = sg; best_b = bd; }
                }
        c->lat_target = best_t; c->lat_stages = best_s; c->lat_bpb = best_b;
        latent_tma_shape(c);
    }
    // 2. FFT passes: rows per block, then columns per block (the Stockham passes; the register-
    // resident passes have one shape, and the S B-in-X variant always runs Stockham rows)
    if (c->fft_impl != 1 || c->xmode == 1) {
        best = 1e30;
        const int old_r = c->fr_rpb;
        int best_r = old_r;
        for (int r : {1, 2, 4, 8}) {
            if (fuse_set_option(c, FUSE_OPT_FFT_ROWS, r) != FUSE_OK) { fuse_reset_error(c); continue; }
            if ((st = time_iterations(c, iters, &t)) != FUSE_OK) return st;
            if (t < best) { best = t; best_r = r; }
        }
        fuse_set_option(c, FUSE_OPT_FFT_ROWS, best_r);
        // the column width applies to the paper's column pass only (the S B-in-X variant's
        // column pass takes its shape from the alias classes)
        if (c->xmode != 1) {
            best = 1e30;
            int best_c = c->fc_cw;
            for (int cw : {2, 4, 8, 16}) {
                if (fuse_set_option(c, FUSE_OPT_FFT_COLS, cw) != FUSE_OK) { fuse_reset_error(c); continue; }
                if ((st = time_iterations(c, iters, &t)) != FUSE_OK) return st;
                if (t < best) { best = t; best_c = cw; }
            }
            fuse_set_option(c, FUSE_OPT_FFT_COLS, best_c);
        }
    }
    drop_graphs(c);
    c->have_state = false;
    c->have_x = false;
    return FUSE_OK;
}

fuse_status fuse_get_option(fuse_ctx* c, int option, long long* value) {
    if (!c || !value) return FUSE_EINVAL;
    switch (option) {
        case FUSE_OPT_PROFILE: *value = c->profile; return FUSE_OK;
        case FUSE_OPT_GRAPH: *value = c->use_graph; return FUSE_OK;
        case FUSE_OPT_LATENT_IMPL: *value = c->lat_impl; return FUSE_OK;
        case FUSE_OPT_LATENT_THREADS: *value = c->lat_target; return FUSE_OK;
        case FUSE_OPT_LATENT_STAGES: *value = c->lat_stages; return FUSE_OK;
        case FUSE_OPT_WAIT_LIMIT: *value = c->wait_limit; return FUSE_OK;
        case FUSE_OPT_HALF_WINDOW: *value = c->half; return FUSE_OK;
        case FUSE_OPT_STATE_FORMAT: *value = c->sfmt; return FUSE_OK;
        case FUSE_OPT_LATENT_BANDS: *value = c->lat_bpb; return FUSE_OK;
        case FUSE_OPT_FFT_ROWS: *value = c->fr_rpb; return FUSE_OK;
        case FUSE_OPT_FFT_COLS: *value = c->fc_cw; return FUSE_OK;
        case FUSE_OPT_GRAD_SEGMENT: *value = c->grad_seg; return FUSE_OK;
        case FUSE_OPT_GRAD_WEIGHTS: *value = c->grad_weights; return FUSE_OK;
        case FUSE_OPT_X_UPDATE: *value = c->xmode; return FUSE_OK;
        case FUSE_OPT_RESIDUALS: *value = c->monitor; return FUSE_OK;
        case FUSE_OPT_SEPARABLE_BLUR: *value = c->sep_blur; return FUSE_OK;
        case FUSE_OPT_FFT_IMPL: *value = c->fft_impl; return FUSE_OK;
        default: return FUSE_EINVAL;
    }
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

fuse_status fuse_batch_create(fuse_batch** out, fuse_ctx* const* ctxs, int n, void* stream) {
    if (!out || !ctxs || n < 1) return FUSE_EINVAL;
    *out = nullptr;
    fuse_ctx* c0 = ctxs[0];
    if (!c0) return FUSE_EINVAL;
    for (int i = 0; i < n; ++i) {
        fuse_ctx* c = ctxs[i];
        if (!c || c->sticky != FUSE_OK) return FUSE_EINVAL;
        if (c->dtype != c0->dtype || c->wdtype != c0->wdtype || c->K != c0->K || c->S != c0->S ||
            c->Ls != c0->Ls || c->bh != c0->bh || c->bw != c0->bw || c->half != c0->half || c->device != c0->device ||
            c->sfmt != c0->sfmt)
            return FUSE_EINVAL;
        if (c->xmode != 0) return FUSE_EUNSUPPORTED;     // batches run the paper's splitting
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return FUSE_EINVAL;
    }
    if (pixel_bucket(c0->Ls) == 0) return FUSE_EUNSUPPORTED;
    fuse_batch* b = new (std::nothrow) fuse_batch();
    if (!b) return FUSE_ENOMEM;
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = (cudaStream_t)stream;
    b->device = c0->device;
    b->dtype = c0->dtype; b->wdtype = c0->wdtype;
    b->K = c0->K; b->S = c0->S; b->Ls = c0->Ls; b->bh = c0->bh; b->bw = c0->bw; b->half = c0->half;
    b->sfmt = c0->sfmt;
    b->same_taps = true;
    for (fuse_ctx* c : b->ctx)
        if (c->htapsT != c0->htapsT) b->same_taps = false;
    b->fc_cw = c0->dtype == FUSE_F64 ? 4 : 8;
    if (cudaSetDevice(b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess || !b->side.create()) {
        cudaGetLastError();
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        b->side.destroy();
        delete b;
        return FUSE_ECUDA;
    }
    for (fuse_ctx* c : b->ctx) c->stream = b->stream;
    fuse_status st = batch_build(b);
    if (st != FUSE_OK) {
        batch_release(b);
        cudaStreamDestroy(b->cap_stream);
        b->side.destroy();
        delete b;
        return st;
    }
    *out = b;
    return FUSE_OK;
}

fuse_status fuse_batch_solve(fuse_batch* b, const void* const* Yl, const void* const* Yh, int iters,
                             void* const* X_out, void* const* Z_out) {
    if (!b || !Yl || !Yh) return FUSE_EINVAL;
    if (b->sticky != FUSE_OK) return FUSE_ESTATE;
    if (iters < 0) return bfail(b, FUSE_EINVAL, "iters must be >= 0");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, FUSE_ECUDA, "cudaSetDevice");
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i) {
        fuse_ctx* c = b->ctx[i];
        if (!Yl[i] || !Yh[i]) return bfail(b, FUSE_EINVAL, "NULL input of a problem");
        if (c->sticky != FUSE_OK || !c->have_weights) return bfail(b, FUSE_ESTATE, "a problem has no weights or holds an error");
        c->stream = b->stream;
        const bool f64 = c->dtype == FUSE_F64;
        fuse_status st = f64 ? Impl<double>::band_mix(c, b->stream, Yl[i], c->D9a, c->Et, c->nl, c->Ll, c->Ls)
                             : Impl<float>::band_mix(c, b->stream, Yl[i], c->D9a, c->Et, c->nl, c->Ll, c->Ls);
        if (st == FUSE_OK)
            st = f64 ? Impl<double>::band_mix(c, b->stream, Yh[i], c->D9b, c->Mh, c->n, c->Lh, c->Ls)
                     : Impl<float>::band_mix(c, b->stream, Yh[i], c->D9b, c->Mh, c->n, c->Lh, c->Ls);
        // with at least one iteration the first batched latent pass takes the state as zero
        if (st == FUSE_OK) st = zero_state(c, b->stream, iters == 0);
        if (st != FUSE_OK) return bfail(b, st, "problem " + std::to_string(i) + ": " + c->err);
        c->have_state = true;
    }
    fuse_status st = batch_run(b, iters, iters > 0);
    if (st != FUSE_OK) return st;
    for (int i = 0; i < n; ++i) {
        fuse_ctx* c = b->ctx[i];
        c->have_x = true;
        const size_t img = c->n * c->Ls * c->esz;
        if (X_out && X_out[i]) BCK(b, cudaMemcpyAsync(X_out[i], c->X, img, cudaMemcpyDeviceToDevice, b->stream));
        if (Z_out && Z_out[i]) {
            const bool f64 = c->dtype == FUSE_F64;
            st = f64 ? Impl<double>::band_mix(c, b->stream, c->X, Z_out[i], c->Emix, c->n, c->Ls, c->Ll)
                     : Impl<float>::band_mix(c, b->stream, c->X, Z_out[i], c->Emix, c->n, c->Ls, c->Ll);
            if (st != FUSE_OK) return bfail(b, st, "problem " + std::to_string(i) + ": " + c->err);
        }
    }
    return FUSE_OK;
}

fuse_status fuse_batch_run_host(fuse_batch* b, const void* const* Yl_h, const void* const* Yh_h,
                                const void* const* G_h, int iters, void* const* X_h, void* const* Z_h) {
    if (!b || !Yl_h || !Yh_h) return FUSE_EINVAL;
    if (b->sticky != FUSE_OK) return FUSE_ESTATE;
    if (iters < 0) return bfail(b, FUSE_EINVAL, "iters must be >= 0");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, FUSE_ECUDA, "cudaSetDevice");
    const int n = (int)b->ctx.size();
    std::vector<const void*> yl(n), yh(n);
    std::vector<void*> xo(n, nullptr), zo(n, nullptr);
    for (int i = 0; i < n; ++i) {
        fuse_ctx* c = b->ctx[i];
        if (!Yl_h[i] || !Yh_h[i]) return bfail(b, FUSE_EINVAL, "NULL input of a problem");
        if (c->sticky != FUSE_OK) return bfail(b, FUSE_ESTATE, "problem " + std::to_string(i) + " holds an error");
        const void* g = G_h ? G_h[i] : nullptr;
        if (!g && c->Lg != c->Lh)
            return bfail(b, FUSE_EINVAL, "problem " + std::to_string(i) + ": guide defaults to Y_h but L_guide != L_h");
        const size_t bl = (size_t)c->Ll * c->nl * c->esz, bhh = (size_t)c->Lh * c->n * c->esz;
        const size_t bg = (size_t)c->Lg * c->n * c->esz;
        const size_t bx = (size_t)c->Ls * c->n * c->esz, bz = (size_t)c->Ll * c->n * c->esz;
        fuse_status st = FUSE_OK;
        if (st == FUSE_OK && !c->sYl) st = dalloc(c, &c->sYl, bl);
        if (st == FUSE_OK && !c->sYh) st = dalloc(c, &c->sYh, bhh);
        if (st == FUSE_OK && g && !c->sG) st = dalloc(c, &c->sG, bg);
        if (st == FUSE_OK && X_h && X_h[i] && !c->sX) st = dalloc(c, &c->sX, bx);
        if (st == FUSE_OK && Z_h && Z_h[i] && !c->sZ) st = dalloc(c, &c->sZ, bz);
        if (st != FUSE_OK) return bfail(b, st, "problem " + std::to_string(i) + ": " + c->err);
        BCK(b, cudaMemcpyAsync(c->sYl, Yl_h[i], bl, cudaMemcpyHostToDevice, b->stream));
        BCK(b, cudaMemcpyAsync(c->sYh, Yh_h[i], bhh, cudaMemcpyHostToDevice, b->stream));
        if (g) BCK(b, cudaMemcpyAsync(c->sG, g, bg, cudaMemcpyHostToDevice, b->stream));
        c->stream = b->stream;
        st = weights_impl(c, g ? c->sG : c->sYh);
        if (st != FUSE_OK) return bfail(b, st, "problem " + std::to_string(i) + ": " + c->err);
        yl[i] = c->sYl;
        yh[i] = c->sYh;
        if (X_h && X_h[i]) xo[i] = c->sX;
        if (Z_h && Z_h[i]) zo[i] = c->sZ;
    }
    fuse_status st = fuse_batch_solve(b, yl.data(), yh.data(), iters, xo.data(), zo.data());
    if (st != FUSE_OK) return st;
    for (int i = 0; i < n; ++i) {
        fuse_ctx* c = b->ctx[i];
        if (xo[i]) BCK(b, cudaMemcpyAsync(X_h[i], xo[i], (size_t)c->Ls * c->n * c->esz, cudaMemcpyDeviceToHost, b->stream));
        if (zo[i]) BCK(b, cudaMemcpyAsync(Z_h[i], zo[i], (size_t)c->Ll * c->n * c->esz, cudaMemcpyDeviceToHost, b->stream));
    }
    return fuse_batch_sync(b);
}

fuse_status fuse_batch_set_option(fuse_batch* b, int option, long long value) {
    if (!b) return FUSE_EINVAL;
    if (b->sticky != FUSE_OK) return FUSE_ESTATE;
    switch (option) {
        case FUSE_OPT_PROFILE: b->profile = value != 0; return FUSE_OK;
        case FUSE_OPT_GRAPH: b->use_graph = value != 0; return FUSE_OK;
        case FUSE_OPT_LATENT_THREADS:
            return batch_set_shape(b, (int)value, b->lat_stages, b->lat_bpb);
        case FUSE_OPT_LATENT_STAGES:
            return batch_set_shape(b, b->lat_target, (int)value, b->lat_bpb);
        case FUSE_OPT_LATENT_BANDS:
            return batch_set_shape(b, b->lat_target, b->lat_stages, (int)value);
        default: return bfail(b, FUSE_EINVAL, "unknown batch option");
    }
}

fuse_status fuse_batch_get_option(fuse_batch* b, int option, long long* value) {
    if (!b || !value) return FUSE_EINVAL;
    switch (option) {
        case FUSE_OPT_PROFILE: *value = b->profile; return FUSE_OK;
        case FUSE_OPT_GRAPH: *value = b->use_graph; return FUSE_OK;
        case FUSE_OPT_LATENT_THREADS: *value = b->lat_target; return FUSE_OK;
        case FUSE_OPT_LATENT_STAGES: *value = b->lat_stages; return FUSE_OK;
        case FUSE_OPT_LATENT_BANDS: *value = b->lat_bpb; return FUSE_OK;
        default: return FUSE_EINVAL;
    }
}

fuse_status fuse_batch_autotune(fuse_batch* b, const void* const* Yl, const void* const* Yh, int iters) {
    if (!b || !Yl || !Yh || iters < 1) return FUSE_EINVAL;
    if (b->sticky != FUSE_OK) return FUSE_ESTATE;
    const bool g = b->use_graph, pr = b->profile;
    b->use_graph = false;
    b->profile = false;
    fuse_status st = fuse_batch_solve(b, Yl, Yh, 0, nullptr, nullptr);   // inputs and zero state
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == FUSE_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = bfail(b, FUSE_ECUDA, "cudaEventCreate");
    double best = 1e30;
    int bt = b->lat_target, bs = b->lat_stages, bb = b->lat_bpb;
    const int threads[] = {128, 160, 192, 256}, stages[] = {6, 8, 12, 16}, bands[] = {1, 2, 4, 8};
    for (int th : threads)
        for (int sg : stages)
            for (int bd : bands) {
                if (st != FUSE_OK) break;
                if (batch_set_shape(b, th, sg, bd) != FUSE_OK) {
                    b->sticky = FUSE_OK;
                    continue;
                }
                st = batch_run(b, 1);
                cudaEventRecord(e0, b->stream);
                if (st == FUSE_OK) st = batch_run(b, iters);
                cudaEventRecord(e1, b->stream);
                float t = 0.f;
                if (st == FUSE_OK && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t < best) {
                    best = t; bt = th; bs = sg; bb = bd;
                }
            }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->use_graph = g;
    b->profile = pr;
    if (st != FUSE_OK) return st;
    return batch_set_shape(b, bt, bs, bb);
}

fuse_status fuse_batch_profile(fuse_batch* b, int which, double* ms, long long* launches, int reset) {
    if (!b) return FUSE_EINVAL;
    BCK(b, cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < b->ev_used; ++i) {
        float t = 0.f;
        BCK(b, cudaEventElapsedTime(&t, b->ev[i].a, b->ev[i].b));
        b->latent_ms += t;
    }
    b->ev_used = 0;
    long long extra = 0;
    for (fuse_ctx* c : b->ctx) extra += c->launches_all;
    if (which == FUSE_K_LATENT) {
        if (ms) *ms = b->latent_ms;
        if (launches) *launches = b->launches_latent;
    } else if (which == FUSE_K_ALL) {
        if (ms) *ms = 0.0;
        if (launches) *launches = b->launches_all + extra;
    } else {
        return bfail(b, FUSE_EINVAL, "unknown kernel group");
    }
    if (reset) {
        b->latent_ms = 0.0; b->launches_latent = 0; b->launches_all = 0;
        for (fuse_ctx* c : b->ctx) c->launches_all = 0;
    }
    return FUSE_OK;
}

fuse_status fuse_batch_sync(fuse_batch* b) {
    if (!b) return FUSE_EINVAL;
    BCK(b, cudaStreamSynchronize(b->stream));
    for (fuse_ctx* c : b->ctx) {
        fuse_status st = fuse_sync(c);
        if (st != FUSE_OK) return bfail(b, st, c->err);
    }
    return FUSE_OK;
}

fuse_status fuse_batch_destroy(fuse_batch* b) {
    if (!b) return FUSE_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    b->side.destroy();
    delete b;
    return FUSE_OK;
}

const char* fuse_batch_last_error(const fuse_batch* b) { return b ? b->err.c_str() : ""; }

fuse_status fuse_reset_error(fuse_ctx* c) {
    if (!c) return FUSE_EINVAL;
    c->sticky = FUSE_OK;
    c->err.clear();
    return FUSE_OK;
}

fuse_status fuse_set_mask(fuse_ctx* c, const void* mask) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (mask && c->d != 1) return fail(c, FUSE_EINVAL, "a sampling mask needs ratio 1");
    if (mask && c->xmode == 1) return fail(c, FUSE_EUNSUPPORTED, "the S B-in-X update needs the regular lattice");
    if (!mask) {
        c->mask = nullptr;
    } else {
        if (!c->mask_buf && (st = dalloc(c, &c->mask_buf, c->n)) != FUSE_OK) return st;
        CK(c, cudaMemcpyAsync(c->mask_buf, mask, c->n, cudaMemcpyDefault, c->stream));
        c->mask = c->mask_buf;
    }
    // the pixel launches carry the mask pointer: drop the captured iteration graph
    drop_graphs(c);
    ++c->epoch;
    return FUSE_OK;
}

fuse_status fuse_conditioning(fuse_ctx* c, double out[3]) {
    if (!c || !out) return FUSE_EINVAL;
    for (int q = 0; q < 3; ++q) out[q] = c->cond[q];
    return FUSE_OK;
}

fuse_status fuse_grad_bytes(fuse_ctx* c, int iters, size_t* bytes) {
    if (!c || !bytes || iters < 0) return FUSE_EINVAL;
    *bytes = grad_bytes(c, iters);
    return FUSE_OK;
}

fuse_status fuse_grad_forward(fuse_ctx* c, const void* Yl, const void* Yh, int iters, void* X_out) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!Yl || !Yh) return fail(c, FUSE_EINVAL, "Y_l or Y_h is NULL");
    if (iters < 0) return fail(c, FUSE_EINVAL, "iters must be >= 0");
    if (!c->have_weights) return FUSE_ESTATE;
    if (pixel_bucket(c->Ls) == 0) return fail(c, FUSE_EUNSUPPORTED, "the reverse pass supports L_s <= 32");
    if (c->sfmt) return fail(c, FUSE_EUNSUPPORTED, "the reverse pass needs the state in the iterate type");
    if (c->xmode) return fail(c, FUSE_EUNSUPPORTED, "the reverse pass follows the paper's splitting");
    return grad_forward_impl(c, Yl, Yh, iters, X_out);
}

fuse_status fuse_grad_backward(fuse_ctx* c, const void* Xbar, const void* Zbar, void* Yl_bar, void* Yh_bar,
                               double* param_bar) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!Xbar && !Zbar) return fail(c, FUSE_EINVAL, "both dL/dX and dL/dZ are NULL");
    return grad_backward_impl(c, Xbar, Zbar, Yl_bar, Yh_bar, param_bar);
}

fuse_status fuse_grad_weights(fuse_ctx* c, void* omega_bar, const void* guide, void* guide_bar) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    return grad_weights_impl(c, omega_bar, guide, guide_bar);
}

fuse_status fuse_grad(fuse_ctx* c, const void* Yl, const void* Yh, int iters, const void* Xbar, const void* Zbar,
                      void* X_out, void* Yl_bar, void* Yh_bar, double* param_bar) {
    fuse_status st = guard(c);
    if (st != FUSE_OK) return st;
    if (!Xbar && !Zbar) return fail(c, FUSE_EINVAL, "both dL/dX and dL/dZ are NULL");
    st = fuse_grad_forward(c, Yl, Yh, iters, X_out);
    if (st != FUSE_OK) return st;
    return grad_backward_impl(c, Xbar, Zbar, Yl_bar, Yh_bar, param_bar);
}

}  // extern "C"
