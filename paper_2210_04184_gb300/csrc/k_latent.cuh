// Fused latent pass of one ADMM iteration: Q update (eq. Qj_main), Sigma dual update
// (eq. dualvar3_main) and the adjoint sum sum_{tau,k} D_{tau k}^T (Q + Sigma) that enters the
// next right-hand side C (Sec. IV-A, after eq. x_linear_system_main).
//
// Exact rewrite used here.  With v = D_{tau k} X - Sigma and mu = lambda2 omega / rho,
//   Q' = S(v, mu) = v - clamp(v, -mu, mu),
//   Sigma' = Sigma - (D_{tau k}X - Q') = -clamp(v, -mu, mu),
//   G = Q' + Sigma' = v - 2 clamp(v, -mu, mu),
// so Q never has to be stored.  The state is kept re-indexed by the source pixel of the
// shift identity D_{tau k}X(i) = D_{tau 0}X(i - k) (Sec. III): Sig'_{tau k}(m) =
// Sigma_{tau k}(m + k).  For a pixel m the pass then needs delta = X(m) - X(m - tau) once
// per tau, the weight omega_tau(m + k) (the threshold is indexed by the output pixel
// i = m + k, eq. regfilt1) and the contiguous stream Sig'_{tau k}(m).
// The adjoint D_{tau k}^T sends +G to pixel i - k = m and -G to m - tau, so with
// H_tau(m) = sum_k G_{tau k}(m + k):
//   R(j) = sum_tau H_tau(j) - sum_tau H_tau(j + tau).
// One block owns rows [y0, y0+Ty) over the full width, one tau1 and one band c, and writes
//   A_{tau1}(m) = sum_{tau2} H_{(tau1,tau2)}(m)          (plane tau1 + S)
//   V_{tau1}(m) = sum_{tau2} H_{(tau1,tau2)}(m + (0,tau2)) (plane (2S+1) + tau1 + S)
// so that R(j) = sum_{tau1} [A_{tau1}(j) - V_{tau1}(j + (tau1, 0))], summed in fixed order by
// the right-hand-side kernel (deterministic, no atomics).
//
// Half-window mode (half = 1): with M Y(i) = -Y(i + tau), D_{-tau,k} = M D_{tau,k}, and the weights
// satisfy omega_{i,-tau} = omega_{i+tau,tau}; the soft threshold is odd, so from zero state
// Sigma_{-tau,k} = M Sigma_{tau,k} at every iteration and, M being orthogonal,
// D_{-tau,k}^T (Q + Sigma)_{-tau,k} = D_{tau,k}^T (Q + Sigma)_{tau,k}.  Only the offsets of
// W+ = {tau1 > 0} U {tau1 = 0, tau2 > 0} are kept and their adjoint sum is counted twice by the
// right-hand-side kernel: the full-window iterates up to summation order, with half the state.
//
// Layouts: X [L_s][H][W]; omega [|W|][H][W]; Sig' [|W| or |W|/2][|P|][L_s][H][W];
// planes [L_s][2(2S+1)][H][W].  Threads: (W/VEC) x Ty, each owning VEC consecutive pixels.
#pragma once
#include "common.cuh"

namespace fuse {

template <typename T, typename WT, int K, int VEC>
__global__ void __launch_bounds__(256)
latent_kernel(const T* __restrict__ X, const WT* __restrict__ omega, const T* Sig, T* Sout,
              T* __restrict__ planes, int H, int W, int Ls, int S, int Ty, T coef, int half) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Hs = reinterpret_cast<T*>(smem_raw);           // [(2S+1)][Ty][W]
    constexpr int PS = 2 * K + 1;
    constexpr int NP = PS * PS;
    const int tpr = W / VEC;
    const int tid = threadIdx.x;
    const int r = tid / tpr;
    const int x0 = (tid - r * tpr) * VEC;
    const int y = blockIdx.x * Ty + r;
    const TauMap tm{S, half};
    const int t1 = tm.t1_of_block(blockIdx.z);
    const int nt2 = tm.nt2(t1);
    const int c = blockIdx.y;
    const bool active = y < H;
    const size_t n = (size_t)H * W;
    const int side = 2 * S + 1;
    const T* Xc = X + (size_t)c * n;
    const size_t kstride = (size_t)Ls * n;

    T Xm[VEC];
    T A[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) { Xm[j] = active ? Xc[(size_t)y * W + x0 + j] : T(0); A[j] = T(0); }

    for (int jt = 0; jt < nt2; ++jt) {
        const int t2 = tm.t2_of(t1, jt);
        T Hacc[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) Hacc[j] = T(0);
        if (active) {
            const int ys = wrap1(y - t1, H);
            T delta[VEC];
#pragma unroll
            for (int j = 0; j < VEC; ++j) delta[j] = Xm[j] - Xc[(size_t)ys * W + wrap1(x0 + j - t2, W)];
            const WT* om = omega + (size_t)tm.w_index(t1, t2) * n;
            const size_t soff = ((size_t)tm.s_index(t1, t2) * NP * Ls + c) * n + (size_t)y * W + x0;
            const vecT<T, VEC>* sp = reinterpret_cast<const vecT<T, VEC>*>(Sig + soff);
            vecT<T, VEC>* so = reinterpret_cast<vecT<T, VEC>*>(Sout + soff);
            const size_t vstride = kstride / VEC;
#pragma unroll
            for (int k1 = -K; k1 <= K; ++k1) {
                // mu for the output pixels i = m + k, k2 in [-K, K]: columns x0-K .. x0+VEC-1+K
                const int yw = wrap1(y + k1, H);
                SymBound<T> mu[VEC + 2 * K];
#pragma unroll
                for (int j = 0; j < VEC + 2 * K; ++j)
                    mu[j] = SymBound<T>::of(coef * (T)wload(om + (size_t)yw * W + wrap1(x0 - K + j, W)));
                // issue the 2K+1 loads of this patch row before any store
                vecT<T, VEC> s[PS];
#pragma unroll
                for (int k2 = 0; k2 < PS; ++k2) s[k2] = ld_stream(sp + (size_t)k2 * vstride);
#pragma unroll
                for (int k2 = 0; k2 < PS; ++k2) {
#pragma unroll
                    for (int j = 0; j < VEC; ++j) {
                        const T u = s[k2].v[j] - delta[j];         // -v
                        const T s2 = mu[j + k2].clamp(u);          // Sigma' = -clamp(v)
                        Hacc[j] += T(2) * s2 - u;                  // G = v + 2 Sigma'
                        s[k2].v[j] = s2;
                    }
                    st_stream(so + (size_t)k2 * vstride, s[k2]);
                }
                sp += (size_t)PS * vstride;
                so += (size_t)PS * vstride;
            }
        }
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            A[j] += Hacc[j];
            Hs[((size_t)(t2 + S) * Ty + r) * W + x0 + j] = Hacc[j];
        }
    }
    __syncthreads();
    if (!active) return;
    T V[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) V[j] = T(0);
    for (int jt = 0; jt < nt2; ++jt) {
        const int t2 = tm.t2_of(t1, jt);
        const T* row = Hs + ((size_t)(t2 + S) * Ty + r) * W;
#pragma unroll
        for (int j = 0; j < VEC; ++j) V[j] += row[wrap1(x0 + j + t2, W)];
    }
    T* pa = planes + ((size_t)c * 2 * side + (t1 + S)) * n + (size_t)y * W + x0;
    T* pv = planes + ((size_t)c * 2 * side + side + (t1 + S)) * n + (size_t)y * W + x0;
    vecT<T, VEC> va, vv;
#pragma unroll
    for (int j = 0; j < VEC; ++j) { va.v[j] = A[j]; vv.v[j] = V[j]; }
    *reinterpret_cast<vecT<T, VEC>*>(pa) = va;
    *reinterpret_cast<vecT<T, VEC>*>(pv) = vv;
}

}  // namespace fuse

// ---------------------------------------------------------------------------------------
// Pipelined form of the same pass (each consumer thread owns VEC pixels; VEC * sizeof(T) is
// 16 or 32 bytes): the latent state is streamed through a shared-memory ring
// by bulk asynchronous copies (cp.async.bulk, 1D TMA), issued by one producer warp, so the
// number of bytes in flight no longer depends on registers.  One chunk = the block's rows of
// one (tau, k) plane of Sig' (Ty*W contiguous elements).  Consumers wait on the chunk's
// `full` barrier, update their VEC elements, store them back with streaming 16-byte stores
// and release the slot through its `empty` barrier (one arrival per consumer warp).
// Every barrier wait is bounded (`limit` polls); a timeout sets bit 1 of *err and the kernel
// still finishes in bounded time.
#include "tma.cuh"

namespace fuse {

// Position, in a row interleaved by VEC (element x at (x mod VEC) tpr + x / VEC, tpr = W / VEC), of
// the element x0 + q (circular in the row) for the thread with x0 = VEC tcol: word
// (q mod VEC) tpr + (tcol + floor(q / VEC)) mod tpr, since W and x0 are multiples of VEC.  One
// wrap suffices: |floor(q / VEC)| <= tpr for the shifts used here (|q| <= S + VEC - 1, W >= 2S + 1).
template <int VEC>
__device__ __forceinline__ int ishift(int tcol, int q, int tpr) {
    static_assert((VEC & (VEC - 1)) == 0, "VEC is a power of two");
    constexpr int LV = VEC == 8 ? 3 : VEC == 4 ? 2 : VEC == 2 ? 1 : 0;
    return (q & (VEC - 1)) * tpr + wrap1(tcol + (q >> LV), tpr);
}

template <typename T, typename WT>
struct LatentArgs {
    const T* X;
    const WT* omega;
    const void* Sig;    // state read (bulk copies), elements of the storage type
    void* Sout;         // state written: Sig itself, or another buffer of the same layout
    T* planes;
    int H, W, Ls, S, Ty, ncons, D;
    T coef;
    int* err;
    unsigned limit;
    int half;
    int bpb;            // bands per block: the ring keeps streaming across them
    int zero_in;        // 1: the entering state is zero (first iteration of a cold solve): nothing
                        // is read, the pass only writes the new state and the adjoint sums
    // monitoring instance only (latent_tma_monitor_kernel): adjoint planes of Q' + Sigma (same
    // layout as `planes`) and one FP64 sum of (Sigma' - Sigma)^2 per block
    T* mplanes;
    double* mpart;
};

__device__ __forceinline__ void consumer_barrier(int ncons) {
    asm volatile("bar.sync 1, %0;" ::"r"(ncons) : "memory");
}

// The weights of one row of the patch window for a thread's VEC pixels: omega at columns
// x0 - K .. x0 + VEC - 1 + K of one weight row (circular), the middle VEC in one aligned vector
// load and the K on each side as single loads.  Loaded one row ahead of its use.
template <typename WT, int VEC, int K>
struct WRow {
    vecT<WT, VEC> mid;
    WT lo[K > 0 ? K : 1], hi[K > 0 ? K : 1];
    __device__ __forceinline__ void load(const WT* __restrict__ row, int x0, int W) {
        mid = *reinterpret_cast<const vecT<WT, VEC>*>(row + x0);
#pragma unroll
        for (int i = 0; i < K; ++i) {
            lo[i] = row[wrap1(x0 - K + i, W)];
            hi[i] = row[wrap1(x0 + VEC + i, W)];
        }
    }
    // weight at column x0 - K + j (j in [0, VEC + 2K))
    __device__ __forceinline__ auto get(int j) const {
        return wconv(j < K ? lo[j] : (j < K + VEC ? mid.v[j - K] : hi[j - K - VEC]));
    }
};

// Block (bx, g, row) of one problem: rows [bx*Ty, bx*Ty + Ty), bands [g*bpb, g*bpb + bpb),
// tau1 row `row`.  The bands are processed one after the other while the producer keeps the
// ring full.  Per band the consumers stage their X values X(m) (Xo) and the row segment
// X(m - (tau1, 0)) (Xs) in shared memory, so delta = X(m) - X(m - tau) comes from shared memory
// for every tau2; per tau2 each consumer adds its H_tau to A in registers and publishes it in one
// of two shared tiles (alternating), and after one named barrier (the producer never waits on it)
// adds the shifted H_tau(m + (0, tau2)) of its row to its entries of the V tile (Vs).
// The shifted tiles (Xs and the H tiles, read at x0 + j -+ tau2 by the thread owning x0 .. x0 +
// VEC - 1) hold each row interleaved: element x of a row at (x mod VEC) tpr + x / VEC, tpr = W /
// VEC, so for a fixed j the threads of a row access consecutive words (the natural layout puts
// them VEC words apart, a VEC-way bank conflict on every such access).
// Shared memory: ring [D][Ty][W] (storage type), then the tiles Xo, Vs, two H tiles, Xs and with
// MON two tiles of the monitoring sums, each [Ty][W] of T (W % 8 == 0 keeps every tile a
// multiple of 32 bytes, so the 16-byte vector accesses stay aligned), then the 2D mbarriers.
// MON (monitoring instance, the last iteration of a solve whose residuals are wanted) also forms
// the adjoint sums of Q' + Sigma = v + Sigma' + Sigma (into args.mplanes) and the block's sum of
// (Sigma' - Sigma)^2 (into args.mpart): the latent parts of the ADMM dual and primal residuals
// (Sec. IV, eq. dualvar3_main: D X - Q' = Sigma - Sigma').
template <typename T, typename WT, int K, int VEC, typename ST, bool MON = false>
__device__ __forceinline__ void latent_tma_body(const LatentArgs<T, WT>& args, int bx, int g, int row,
                                                unsigned char* smem_tma) {
    const T* __restrict__ X = args.X;
    const WT* __restrict__ omega = args.omega;
    const ST* Sig = static_cast<const ST*>(args.Sig);
    ST* Sout = static_cast<ST*>(args.Sout);
    T* __restrict__ planes = args.planes;
    const int H = args.H, W = args.W, Ls = args.Ls, S = args.S, Ty = args.Ty, ncons = args.ncons, D = args.D;
    const T coef = args.coef;
    int* __restrict__ err = args.err;
    const unsigned limit = args.limit;
    const int half = args.half;
    constexpr int PS = 2 * K + 1;
    constexpr int NP = PS * PS;
    const int side = 2 * S + 1;
    const int tile = Ty * W;
    ST* ring = reinterpret_cast<ST*>(smem_tma);               // [D][Ty][W] of the storage type
    T* Xo = reinterpret_cast<T*>(ring + (size_t)D * tile);    // [Ty][W]
    T* Vs = Xo + tile;                                        // [Ty][W]
    T* Hb = Vs + tile;                                        // [2][Ty][W]
    T* Xs = Hb + (size_t)2 * tile;                            // [Ty][W]
    T* Mb = Xs + tile;                                        // MON only: [2][Ty][W]
    constexpr int NT = MON ? 7 : 5;
    uint64_t* full = reinterpret_cast<uint64_t*>(Xo + (size_t)NT * tile);
    uint64_t* empty = full + D;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x;
    const int tpr = W / VEC;
    const int y0 = bx * Ty;
    const int rows = min(Ty, H - y0);
    const TauMap tm{S, half};
    const int t1 = tm.t1_of_block(row);
    const size_t n = (size_t)H * W;
    const int nt2 = tm.nt2(t1);
    const int c0 = g * args.bpb;
    const int nb = min(args.bpb, Ls - c0);
    const int per_band = nt2 * NP;
    const int nq = nb * per_band;
    const unsigned bytes = (unsigned)(rows * W * (int)sizeof(ST));
    const bool zin = args.zero_in != 0;

    if (tid == 0) {
        for (int s = 0; s < D; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (unsigned)(ncons / 32));
        }
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();

    if (tid >= ncons) {
        // ---------------- producer warp: one lane issues the bulk copies ----------------
        if (tid == ncons && !zin) {
            const uint64_t pol = l2_evict_first_policy();
            int issued = 0;
            for (int q = 0; q < nq; ++q) {
                if (s_abort) break;                 // never re-arm a barrier after a timeout
                const int slot = q % D;
                if (q >= D && !mbar_wait(&empty[slot], (unsigned)((q / D - 1) & 1), limit, err, 1)) {
                    s_abort = 1;
                    break;
                }
                const int item = q / per_band, rem = q - item * per_band;
                const int j = rem / NP, kidx = rem - j * NP;
                const int t2 = tm.t2_of(t1, j);
                const ST* src = Sig + ((size_t)(tm.s_index(t1, t2) * NP + kidx) * Ls + (c0 + item)) * n +
                               (size_t)y0 * W;
                mbar_arrive_expect_tx(&full[slot], bytes);
                tma_load_1d(ring + (size_t)slot * tile, src, bytes, &full[slot], pol);
                issued = q + 1;
            }
            // drain: no bulk copy of this block may still be in flight when it exits; copies of
            // valid memory always land, so the bound here is generous whatever `limit` is
            const unsigned dlim = limit > (1u << 20) ? limit : (1u << 20);
            for (int q = issued > D ? issued - D : 0; q < issued; ++q)
                if (!mbar_wait(&full[q % D], (unsigned)((q / D) & 1), dlim, err, 1)) break;
        }
        return;
    }

    // ---------------- consumers (threads >= tpr*Ty own no pixels) ----------------
    const int lane = tid & 31;
    const int r = tid / tpr;
    const int x0 = (tid - r * tpr) * VEC;
    const int y = y0 + r;
    const bool owner = tid < tpr * Ty;
    const int tcol = x0 / VEC;                           // the thread's word in each interleaved row
    const bool active = owner && r < rows;
    const size_t pix = (size_t)y * W + x0;
    const size_t kstride = (size_t)Ls * n;
    const size_t xsrow = (size_t)wrap1(y - t1, H) * W;   // row of X(m - tau) (active threads)
    int slot = 0;
    unsigned par = 0;
    unsigned lim = limit;                                // 64 polls once a wait has timed out
    int hb = 0;                                          // H tile written next
    double dsq = 0.0;                                    // MON only: sum of (Sigma' - Sigma)^2
    for (int item = 0; item < nb; ++item) {
        const int c = c0 + item;
        const T* Xc = X + (size_t)c * n;
        T* xo = Xo + (size_t)r * W + x0;
        T* vs = Vs + (size_t)r * W + x0;
        if (active) {
            T xr[VEC];
            vload<T, VEC>(Xc + pix, xr);
            vstore<T, VEC>(xo, xr);
            vload<T, VEC>(Xc + xsrow + x0, xr);
#pragma unroll
            for (int j = 0; j < VEC; ++j) Xs[(size_t)r * W + j * tpr + tcol] = xr[j];
#pragma unroll
            for (int j = 0; j < VEC; ++j) xr[j] = T(0);
            vstore<T, VEC>(vs, xr);
        }
        consumer_barrier(ncons);                 // Xs holds the band's shifted rows
        T A[VEC];
        T A2[MON ? VEC : 1], V2[MON ? VEC : 1];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            A[j] = T(0);
            if constexpr (MON) { A2[j] = T(0); V2[j] = T(0); }
        }
        WRow<WT, VEC, K> wr;
        if (active) wr.load(omega + (size_t)tm.w_index(t1, tm.t2_of(t1, 0)) * n + (size_t)wrap1(y - K, H) * W, x0, W);
        for (int jt = 0; jt < nt2; ++jt) {
            const int t2 = tm.t2_of(t1, jt);
            T Hacc[VEC], delta[VEC];
            T Macc[MON ? VEC : 1];
            if (active) vload<T, VEC>(xo, delta);
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
                Hacc[j] = T(0);
                if constexpr (MON) Macc[j] = T(0);
                delta[j] = active ? delta[j] - Xs[(size_t)r * W + ishift<VEC>(tcol, j - t2, tpr)] : T(0);
            }
            const WT* om = omega + (size_t)tm.w_index(t1, t2) * n;
            const WT* om_next = jt + 1 < nt2 ? omega + (size_t)tm.w_index(t1, tm.t2_of(t1, jt + 1)) * n : om;
            ST* gp = Sout + ((size_t)tm.s_index(t1, t2) * NP * Ls + c) * n + pix;
#pragma unroll
            for (int k1 = 0; k1 < PS; ++k1) {
                if constexpr (std::is_same<ST, T>::value) {
                    SymBound<T> mu[VEC + 2 * K];
#pragma unroll
                    for (int j = 0; j < VEC + 2 * K; ++j) mu[j] = SymBound<T>::of(active ? coef * (T)wr.get(j) : T(0));
                    // the next weight row: row k1 + 1, or the first row of the next tau2
                    if (active) {
                        if (k1 + 1 < PS) wr.load(om + (size_t)wrap1(y + k1 + 1 - K, H) * W, x0, W);
                        else if (jt + 1 < nt2) wr.load(om_next + (size_t)wrap1(y - K, H) * W, x0, W);
                    }
#pragma unroll
                    for (int k2 = 0; k2 < PS; ++k2) {
                        if (!zin && !mbar_wait(&full[slot], par, lim, err, 1)) {
                            s_abort = 1;
                            lim = 64u;
                        }
                        if (active) {
                            T sv[VEC];
                            if (zin) {
#pragma unroll
                                for (int j = 0; j < VEC; ++j) sv[j] = T(0);
                            } else {
                                vload<T, VEC>(ring + (size_t)slot * tile + (size_t)r * W + x0, sv);
                            }
#pragma unroll
                            for (int j = 0; j < VEC; ++j) {
                                const T u = sv[j] - delta[j];
                                const T s2 = mu[j + k2].clamp(u);
                                Hacc[j] += T(2) * s2 - u;
                                if constexpr (MON) {
                                    Macc[j] += s2 + sv[j] - u;              // Q' + Sigma
                                    const double dd = (double)(s2 - sv[j]);
                                    dsq += dd * dd;
                                }
                                sv[j] = s2;
                            }
                            vstore_stream<T, VEC>(gp, sv);
                        }
                        if (!zin) {
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&empty[slot]);
                        }
                        gp += kstride;
                        if (++slot == D) { slot = 0; par ^= 1u; }
                    }
                } else {
                    // 16-bit fixed point (see FixedCode): the update runs in code units of mu/32767,
                    // where the clamp bounds are +-32767 and the new code is the clamped value
                    // rounded by one addition; G returns to real units through mu/32767.  Per
                    // weight column: inv = 32767/mu (code units per real unit), sc = mu/32767.
                    static_assert(VEC == 8, "one 16-byte group of codes per thread and chunk");
                    float inv[VEC + 2 * K], sc[VEC + 2 * K];
#pragma unroll
                    for (int j = 0; j < VEC + 2 * K; ++j) {
                        const float m = active ? fmaxf(coef * (float)wr.get(j), FixedCode::kMinMu) : 1.0f;
                        inv[j] = __fdividef(FixedCode::kLevels, m);
                        sc[j] = m * FixedCode::kStep;
                    }
                    if (active) {
                        if (k1 + 1 < PS) wr.load(om + (size_t)wrap1(y + k1 + 1 - K, H) * W, x0, W);
                        else if (jt + 1 < nt2) wr.load(om_next + (size_t)wrap1(y - K, H) * W, x0, W);
                    }
#pragma unroll
                    for (int k2 = 0; k2 < PS; ++k2) {
                        if (!zin && !mbar_wait(&full[slot], par, lim, err, 1)) {
                            s_abort = 1;
                            lim = 64u;
                        }
                        if (active) {
                            // code 0 stands for 0
                            const int4 w = zin ? make_int4(0, 0, 0, 0)
                                               : *reinterpret_cast<const int4*>(ring + (size_t)slot * tile + (size_t)r * W + x0);
                            const uint32_t wd[4] = {(uint32_t)w.x, (uint32_t)w.y, (uint32_t)w.z, (uint32_t)w.w};
                            uint32_t out[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                // the two codes of a word are updated together with the paired
                                // FP32 instructions (same rounding as the scalar ones)
                                const int j0 = 2 * h, j1 = 2 * h + 1;
                                const float2 q = FixedCode::decode2(wd[h]);
                                const float2 uc = __ffma2_rn(make_float2(-delta[j0], -delta[j1]),
                                                             make_float2(inv[j0 + k2], inv[j1 + k2]), q);  // Sigma - D X
                                const float2 s2c = make_float2(fminf(fmaxf(uc.x, -FixedCode::kLevels), FixedCode::kLevels),
                                                               fminf(fmaxf(uc.y, -FixedCode::kLevels), FixedCode::kLevels));
                                const float2 g2 = __ffma2_rn(make_float2(2.0f, 2.0f), s2c, make_float2(-uc.x, -uc.y));
                                const float2 hacc = __ffma2_rn(g2, make_float2(sc[j0 + k2], sc[j1 + k2]),
                                                               make_float2(Hacc[j0], Hacc[j1]));
                                Hacc[j0] = hacc.x;
                                Hacc[j1] = hacc.y;
                                out[h] = FixedCode::pack2(s2c);
                            }
                            __stcs(reinterpret_cast<int4*>(gp), make_int4((int)out[0], (int)out[1], (int)out[2], (int)out[3]));
                        }
                        if (!zin) {
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&empty[slot]);
                        }
                        gp += kstride;
                        if (++slot == D) { slot = 0; par ^= 1u; }
                    }
                }
            }
            // A += H_tau; publish H_tau so the row can form V(m) += H_tau(m + (0, tau2))
            T* ht = Hb + (size_t)hb * tile + (size_t)r * W;
            T* mt = Mb + (size_t)hb * tile + (size_t)r * W;
            if (owner) {
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    A[j] += Hacc[j];
                    ht[j * tpr + tcol] = Hacc[j];
                    if constexpr (MON) {
                        A2[j] += Macc[j];
                        mt[j * tpr + tcol] = Macc[j];
                    }
                }
            }
            // the other H tile was last read before this barrier's previous crossing
            consumer_barrier(ncons);
            if (active) {
                T v[VEC];
                vload<T, VEC>(vs, v);
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    const int e = ishift<VEC>(tcol, j + t2, tpr);
                    v[j] += ht[e];
                    if constexpr (MON) V2[j] += mt[e];
                }
                vstore<T, VEC>(vs, v);
            }
            hb ^= 1;
        }
        if (active) {
            T v[VEC];
            vload<T, VEC>(vs, v);
            vstore<T, VEC>(planes + ((size_t)c * 2 * side + (t1 + S)) * n + pix, A);
            vstore<T, VEC>(planes + ((size_t)c * 2 * side + side + (t1 + S)) * n + pix, v);
            if constexpr (MON) {
                vstore<T, VEC>(args.mplanes + ((size_t)c * 2 * side + (t1 + S)) * n + pix, A2);
                vstore<T, VEC>(args.mplanes + ((size_t)c * 2 * side + side + (t1 + S)) * n + pix, V2);
            }
        }
        // Xs is rewritten by the next band only after every thread has crossed the last tau2's
        // barrier, that is after every read of it (Xo and Vs are read by their owner only)
    }
    if constexpr (MON) {
        // the block's sum of (Sigma' - Sigma)^2 over its consumers, in a fixed order
        __shared__ double s_red[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsq += __shfl_down_sync(0xffffffffu, dsq, o);
        if (lane == 0) s_red[tid >> 5] = dsq;
        consumer_barrier(ncons);
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < ncons / 32; ++w) t += s_red[w];
            args.mpart[blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)] = t;
        }
    }
}

// Register cap: 112 with the state in the iterate type (2 blocks of 288 threads, or 3 of 192, fit
// the 64K registers); 96 with the 16-bit state, which is latency-bound rather than DRAM-bound and
// gains from resident warps (measured at hsms_256: 0.80 ms per launch at 96, 0.92 at 112 and at
// 80, where it spills).
template <typename ST>
constexpr int latent_max_regs() { return sizeof(ST) == 2 ? 96 : 112; }

template <typename T, typename WT, int K, int VEC, typename ST = T>
__global__ void __maxnreg__(latent_max_regs<ST>()) latent_tma_kernel(LatentArgs<T, WT> args) {
    extern __shared__ __align__(128) unsigned char smem_tma[];
    latent_tma_body<T, WT, K, VEC, ST>(args, blockIdx.x, blockIdx.y, blockIdx.z, smem_tma);
}

// The monitoring instance (state in the iterate type): the same update, plus the latent parts of
// the ADMM residuals (see latent_tma_body); needs (2S+1) Ty W more elements of shared memory.
template <typename T, typename WT, int K, int VEC>
__global__ void __launch_bounds__(288, 1) latent_tma_monitor_kernel(LatentArgs<T, WT> args) {
    extern __shared__ __align__(128) unsigned char smem_tma[];
    latent_tma_body<T, WT, K, VEC, T, true>(args, blockIdx.x, blockIdx.y, blockIdx.z, smem_tma);
}

// One launch over many problems (batched uneven sizes): blocks are mapped to (problem, block)
// by the segment table; every problem's launch shape fits the common block size and shared
// memory size of the launch.  zero_in applies to every problem (see LatentArgs).
template <typename T, typename WT, int K, int VEC, typename ST = T>
__global__ void __maxnreg__(latent_max_regs<ST>())
latent_tma_batch_kernel(const LatentArgs<T, WT>* __restrict__ args, const Segment* __restrict__ seg, int nseg,
                        int zero_in) {
    extern __shared__ __align__(128) unsigned char smem_tma[];
    int prob, bx, by, bz;
    segment_of_block(seg, nseg, blockIdx.x, &prob, &bx, &by, &bz);
    LatentArgs<T, WT> a = args[prob];
    a.zero_in = zero_in;
    latent_tma_body<T, WT, K, VEC, ST>(a, bx, by, bz, smem_tma);
}

}  // namespace fuse
