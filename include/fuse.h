/* fuse.h — C-ABI of the GB300 NLPR multiband-fusion solver (libfuse.so).
 *
 * The library solves
 *     min_X  1/2 ||Y_l - S B X E||^2 + lambda1/2 ||Y_h - X E R||^2 + lambda2 phi(X)
 * (Sec. I-A eq. mainoptim) with the nonlocal patch regulariser
 *     phi(X) = sum_i sum_{tau in W} omega_{i tau} ||P_{i tau}(X)||_1        (Sec. II-B eq. reg1)
 * by the ADMM of Sec. IV on the splitting P1 = B X, P2 = X, Q_{tau k} = D_{tau k} X
 * (eq. fusionoptim).  Every iteration is: FFT solve of the X system (eqs.
 * x_linear_system_main, inv), the per-pixel P1/P2 closed forms (eqs. Qh_update,
 * Qm_update), soft thresholding of the latent variables (eq. Qj_main) and the dual
 * updates (eqs. dualvar1_main..dualvar3_main).  The guide weights omega come once from
 * patch distances on the high-resolution guide (eq. wts).
 *
 * Conventions (all entry points):
 *   - Images are planar, band-major, contiguous: band c of an H x W image with L bands
 *     starts at element c*H*W, pixel (i1, i2) is element i1*W + i2 (i1 = row).
 *   - Device pointers must be CUDA device memory of the current device; host pointers
 *     are ordinary (preferably pinned) host memory.  Element type is the context's
 *     dtype (FUSE_F32 -> float, FUSE_F64 -> double) unless stated otherwise.
 *   - Work is issued asynchronously on the context's stream unless stated otherwise.
 *   - Indices are circular (periodic boundary conditions, Sec. II-B).
 *   - The search window is W = [-S, S]^2 without (0, 0), ordered row-major
 *     (tau1 outer); the patch is P = [-K, K]^2, row-major.  |W| = (2S+1)^2 - 1.
 *   - The soft threshold is mu = lambda2 * omega / rho (eq. Qj_main).
 *   - Every call returns a fuse_status; no C++ exception crosses this boundary.  An
 *     error is recorded in the context (sticky until fuse_reset_error) and its text is
 *     available from fuse_last_error.  Calls on a context holding an error return
 *     FUSE_ESTATE without doing work.
 *   - The caller owns every buffer it passes; the library owns everything it allocates
 *     inside a context and frees it in fuse_destroy.
 */
#ifndef FUSE_H
#define FUSE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fuse_status {
    FUSE_OK = 0,
    FUSE_EINVAL = 1,        /* bad argument (null pointer, size, parameter range) */
    FUSE_ENOMEM = 2,        /* device or host allocation failed */
    FUSE_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    FUSE_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    FUSE_ENONFINITE = 5,    /* a non-finite value was detected in a monitored quantity */
    FUSE_ESTATE = 6,        /* call not valid in the context's state (sticky error, no weights) */
    FUSE_EUNSUPPORTED = 7   /* valid request the library does not support (e.g. FFT size) */
} fuse_status;

typedef enum fuse_dtype {
    FUSE_F32 = 0,
    FUSE_F64 = 1,
    FUSE_BF16 = 2           /* weights only */
} fuse_dtype;

/* Sizes of one problem (Sec. I-A): the image is H x W (n_h = H*W pixels, H = p,
 * W = q rows/columns of the periodic domain); Y_l has L_l bands on the (H/ratio) x
 * (W/ratio) lattice, Y_h has L_h bands, X has L_s bands (Z = X E, E is L_s x L_l);
 * the guide passed to fuse_weights has L_guide bands. */
typedef struct fuse_geometry {
    int H, W;
    int L_l, L_h, L_s;
    int L_guide;
} fuse_geometry;

typedef struct fuse_ctx fuse_ctx;

/* Options for fuse_set_option. */
enum {
    FUSE_OPT_PROFILE = 1,        /* 1: time every latent-pass launch with CUDA events (direct
                                    launches, no graph) */
    FUSE_OPT_GRAPH = 2,          /* 1 (default): the whole iteration loop of a solve is one
                                    captured CUDA graph (up to 256 iterations per graph; longer
                                    solves replay it and one graph for the remainder), captured
                                    on first use and kept while the launch configuration holds;
                                    0: direct launches */
    FUSE_OPT_LATENT_IMPL = 3,    /* latent pass: 1 (default) bulk-copy ring, 0 register-staged loads */
    FUSE_OPT_LATENT_THREADS = 4, /* consumer threads per latent block, 32..256 (default 128;
                                    256 in batches) */
    FUSE_OPT_LATENT_STAGES = 5,  /* ring slots of the bulk-copy latent pass, 2..32 (default 6) */
    FUSE_OPT_WAIT_LIMIT = 6,     /* polls before a device barrier wait gives up (default 2^22) */
    FUSE_OPT_HALF_WINDOW = 7,    /* 1 (default): keep the latent state for one offset of each
                                    +-tau pair (exact by the window symmetry, half the state);
                                    0: full window.  Switching reallocates the state and clears it. */
    FUSE_OPT_LATENT_BANDS = 8,   /* bands streamed by one latent block, 1..64 (default 1;
                                    2 in batches) */
    FUSE_OPT_FFT_ROWS = 9,       /* rows per block of the row FFT passes: 1, 2, 4 or 8 */
    FUSE_OPT_FFT_COLS = 10,      /* columns per block of the column FFT pass: power of 2 <= 32 */
    FUSE_OPT_GRAD_SEGMENT = 11,  /* iterations per checkpointed segment of fuse_grad_forward
                                    (default 0: one segment, every iteration taped) */
    FUSE_OPT_GRAD_WEIGHTS = 12,  /* 1: fuse_grad_backward also accumulates dL/domega for
                                    fuse_grad_weights (one more read of the state per reverse
                                    iteration); default 0 */
    FUSE_OPT_STATE_FORMAT = 13,  /* storage of the latent state: 0 (default) the iterate type;
                                    1 = 16-bit fixed point relative to each entry's threshold
                                    (|Sigma'| <= mu always, so q = rint(32767 Sigma'/mu) stands
                                    for q mu / 32767; absolute error <= mu/65534 per entry, half
                                    the state bytes).  F32 contexts with the bulk-copy latent
                                    pass (W % 8 == 0) only; not with the reverse pass.  Switching
                                    reallocates the state and clears it.  A batch takes the
                                    format of its contexts (all the same). */
    FUSE_OPT_X_UPDATE = 14,      /* X update: 0 (default) the paper's splitting (P1 = B X, the X
                                    system diagonal in the DFT basis, eq. inv); 1 = a variant that
                                    is not the paper's: only P2 = X and Q = D X are split, so the X
                                    system keeps the data term,
                                      (I + sum D^T D + eps/rho B^T S^T S B) X
                                        = B^T S^T Y_l E^T / rho + P2 + Lambda2 + sum D^T (Q + Sigma),
                                    solved per alias class of d^2 DFT frequencies in closed form
                                    (diagonal plus rank one; FUSE-type direct solve of the S B
                                    term).  Same objective and limit, other iterates; P1 and
                                    Lambda1 are unused.  Needs the regular lattice (no mask),
                                    E E^T = eps I (orthonormal rows up to a scale, relative
                                    deviation <= 1e-6) and H, W with 2H+1 complex values per
                                    column fitting shared memory; not with the reverse pass or a
                                    batch (FUSE_EUNSUPPORTED).  Switching clears the ADMM state. */
    FUSE_OPT_RESIDUALS = 15,     /* 1: every fuse_solve with iters >= 1 runs its last iteration as a
                                    monitored one (directly launched, about 1.5 times the work of
                                    an iteration) whose ADMM residual norms fuse_residuals returns;
                                    0 (default): off.  Needs the bulk-copy latent pass, the state in
                                    the iterate type and the paper's splitting (FUSE_EUNSUPPORTED
                                    otherwise).  The first switch to 1 allocates 4 images and 2
                                    adjoint-plane arrays of workspace. */
    FUSE_OPT_SEPARABLE_BLUR = 16, /* 1 (default): a square blur whose taps factor as
                                    b(u, v) = cu(u) cv(v) (to 1e-13 of the largest tap, checked at
                                    fuse_init; a sampled Gaussian does) is applied as a horizontal
                                    and a vertical pass (2B multiply-adds per output instead of
                                    B^2; the same operator up to rounding; W % 4 == 0, else the
                                    2D stencil); 0: always the 2D stencil.  A batch follows its
                                    first context. */
    FUSE_OPT_FFT_IMPL = 17       /* DFT solve of the X system: 1 = register-resident passes (one
                                    warp per line, exchanges by warp shuffles; default when H and
                                    W are 32 P with P in {1, 2, 3, 4, 5, 6, 8, 10, 12, 16});
                                    0 = shared-memory Stockham passes (any H, W factoring into 2,
                                    3, 5; FUSE_OPT_FFT_ROWS / FFT_COLS shape them).  Both compute
                                    the same DFT up to rounding.  1 on other sizes:
                                    FUSE_EUNSUPPORTED.  The variant FUSE_OPT_X_UPDATE = 1 always
                                    uses the Stockham passes.  In a batch every problem keeps the
                                    form its context had when the batch was created. */
};

/* Kernel groups for fuse_profile. */
enum {
    FUSE_K_ALL = 0,         /* launch count of every kernel issued by the library */
    FUSE_K_LATENT = 1       /* the fused latent pass (eqs. Qj_main, dualvar3_main, D^T sum) */
};

/* Bytes of device memory fuse_init would allocate for this problem (state in the default
 * half-window mode, weights, FFT buffers and constants).  No device work.  Errors: FUSE_EINVAL, FUSE_EUNSUPPORTED. */
fuse_status fuse_workspace_bytes(const fuse_geometry* g, int K, int S, int ratio,
                                 fuse_dtype dtype, fuse_dtype wdtype, size_t* bytes);

/* Create a solver context (Sec. IV set-up).
 *   g        problem sizes; H and W divisible by `ratio`, H and W factor into 2, 3, 5,
 *            2(K+S)+1 <= min(H, W), W a multiple of 4 (FUSE_F32) or 2 (FUSE_F64).
 *   blur     host, bh x bw row-major (bh, bw odd, bh <= H, bw <= W): the kernel b of B,
 *            centred: blur[a*bw + c] = b(a - bh/2, c - bw/2); B X(i) = sum_j b(j) X(i - j)
 *            with circular indices (Sec. I-A).
 *   ratio    decimation factor d of S: S keeps pixels with i1 = i2 = 0 (mod d).
 *   R        host, L_l x L_h row-major (spectral response, Y_h = Z R).
 *   E        host, L_s x L_l row-major (subspace basis, Z = X E); NULL means E = I
 *            (then L_s must equal L_l).
 *   K, S     patch half-size (|P| = (2K+1)^2, 0 <= K <= 3) and search half-size (S >= 1).
 *   lambda1, lambda2, rho, h   parameters of eqs. mainoptim, wts (lambda1, rho, h > 0,
 *            lambda2 >= 0).
 *   dtype    FUSE_F32 or FUSE_F64: arithmetic and storage type of the iterates.
 *   wdtype   storage type of omega: FUSE_BF16 or FUSE_F32 with FUSE_F32, FUSE_F64 with
 *            FUSE_F64.
 *   stream   cudaStream_t (as void*) on which all later work is issued; NULL = legacy
 *            default stream.
 * Host arrays are copied; the caller keeps ownership.  On success *out receives the
 * context (free with fuse_destroy).  The per-frequency factor of eq. inv and the
 * L_s x L_s inverses of eqs. Qh_update and Qm_update are computed here in FP64 on the
 * host.  Errors: FUSE_EINVAL, FUSE_EUNSUPPORTED, FUSE_ENOMEM, FUSE_ECUDA. */
fuse_status fuse_init(fuse_ctx** out, const fuse_geometry* g, const double* blur, int bh, int bw,
                      int ratio, const double* R, const double* E, int K, int S,
                      double lambda1, double lambda2, double rho, double h,
                      fuse_dtype dtype, fuse_dtype wdtype, void* stream);

/* Free every resource of the context (synchronises its stream first).  NULL is a no-op. */
fuse_status fuse_destroy(fuse_ctx* ctx);

/* Change the stream used by later calls. */
fuse_status fuse_set_stream(fuse_ctx* ctx, void* stream);

/* Guide weights omega_{i tau} = exp(-||P_{i tau}(G)||_2^2 / h^2) (Sec. II-B eq. wts) for every
 * pixel i and tau in W, from the device guide G [L_guide][H][W] (dtype).  Stored in the
 * context as [|W|][H][W] of wdtype.  Must precede fuse_solve.  Errors: FUSE_EINVAL, FUSE_ECUDA. */
fuse_status fuse_weights(fuse_ctx* ctx, const void* guide_dev);

/* Replace the stored weights with w_dev [|W|][H][W] of the context's wdtype (device). */
fuse_status fuse_set_weights(fuse_ctx* ctx, const void* w_dev);

/* Copy the stored weights into w_dev [|W|][H][W] of the context's wdtype (device). */
fuse_status fuse_get_weights(fuse_ctx* ctx, void* w_dev);

/* Run `iters` ADMM iterations (Sec. IV; order X, P1, P2, Q, duals).
 *   Yl_dev   [L_l][H/ratio][W/ratio] (device, dtype)   low-resolution image Y_l
 *   Yh_dev   [L_h][H][W] (device, dtype)               high-resolution image Y_h
 *   iters    >= 0
 *   warm     0: start from zero P1, P2, Q, Lambda1, Lambda2, Sigma (all zero);
 *            1: continue from the state left by the previous fuse_solve/fuse_set_state.
 *   X_out    nullable, [L_s][H][W] (device, dtype): X after the last iteration
 *            (zero when iters == 0 from a zero start).
 *   Z_out    nullable, [L_l][H][W] (device, dtype): Z = X E.
 * Asynchronous on the context stream.  Errors: FUSE_EINVAL, FUSE_ESTATE (no weights), FUSE_ECUDA. */
fuse_status fuse_solve(fuse_ctx* ctx, const void* Yl_dev, const void* Yh_dev, int iters, int warm,
                       void* X_out, void* Z_out);

/* End-to-end call on HOST buffers: copies Y_l, Y_h (and the guide; NULL = use Y_h) to the
 * device, computes the weights, runs fuse_solve from a zero start and copies X and/or Z back
 * (each nullable).  Synchronous: returns after the results are in host memory.  Device
 * staging buffers are allocated on first use and kept by the context.  Sizes and types as in
 * fuse_solve; guide_host [L_guide][H][W].  Errors: as fuse_weights and fuse_solve, and
 * FUSE_EINVAL when the guide is NULL but L_guide != L_h. */
fuse_status fuse_run_host(fuse_ctx* ctx, const void* Yl_host, const void* Yh_host,
                          const void* guide_host, int iters, void* X_host, void* Z_host);

/* Objective terms at the current X (after a fuse_solve): out[0] = 1/2||Y_l - S B X E||^2,
 * out[1] = lambda1/2 ||Y_h - X E R||^2, out[2] = lambda2 phi(X) (eq. mainoptim; eq. reg1),
 * out[3] = ||X||_F^2.  Y_l, Y_h as in fuse_solve.  Synchronous; sums in FP64.
 * Errors: FUSE_ESTATE (no solve yet), FUSE_ENONFINITE (a term is not finite). */
fuse_status fuse_objective(fuse_ctx* ctx, const void* Yl_dev, const void* Yh_dev, double out[4]);

/* ADMM residual norms of the last iteration of the last fuse_solve, which must have run with
 * FUSE_OPT_RESIDUALS = 1 (else FUSE_ESTATE; also after any later call that changed inputs or
 * state).  In the scaled form of the splitting of eq. fusionoptim (A X = z, A = (B; I; D_{tau k}),
 * z = (P1, P2, Q), Sec. IV), for the iteration (X, z) -> (X', z'):
 *   out[0] = primal ||A X' - z'|| = sqrt(||B X' - P1'||^2 + ||X' - P2'||^2 + sum ||D X' - Q'||^2),
 *            which by the dual updates (eqs. dualvar1_main..dualvar3_main) is the change of the
 *            scaled duals ||(Lambda1, Lambda2, Sigma) - (Lambda1', Lambda2', Sigma')||;
 *   out[1] = dual rho ||A^T (z' - z)|| = rho ||B^T (P1' - P1) + (P2' - P2) + sum D^T (Q' - Q)||,
 * over the full search window, summed in FP64 (the paper monitors the objective; these are the
 * standard ADMM stopping quantities).  Synchronous.  Errors: FUSE_ESTATE, FUSE_EINVAL (NULL),
 * FUSE_ENONFINITE (a norm is not finite: the iterates diverged or an input held a NaN). */
fuse_status fuse_residuals(fuse_ctx* ctx, double out[2]);

/* General sampling operator: S keeps the pixels where mask is nonzero instead of the regular
 * lattice (for example a random inpainting mask).  Needs ratio 1 (FUSE_EINVAL otherwise); Y_l
 * is then given at full resolution [L_l][H][W] and its values off the mask do not enter.  S^T S
 * is diagonal either way, so eq. Qh_update and the X update of eq. inv are unchanged; the
 * objective's data term and the reverse pass use the same S.
 *   mask  [H][W] uint8 (host or device; copied, cudaMemcpyDefault), NULL = back to the lattice.
 * Asynchronous on the context stream.  A batch takes its contexts' masks when it is created.
 * Errors: FUSE_EINVAL, FUSE_ENOMEM, FUSE_ECUDA. */
fuse_status fuse_set_mask(fuse_ctx* ctx, const void* mask);

/* Spectral condition numbers of the linear systems the iterations solve, computed in FP64 at
 * fuse_init (host only, no device work):
 *   out[0]  A = I + B^T B + sum_{tau,k} D_{tau k}^T D_{tau k} (eq. x_linear_system_main),
 *           diagonal in the DFT basis: max/min of its eigenvalues 1 + |b^|^2 + |P| sum (2 - 2cos)
 *   out[1]  E E^T + rho I (eq. Qh_update)
 *   out[2]  I + lambda1/rho E R R^T E^T, the inverse of F (eq. Qm_update)
 * The iterate-type arithmetic needs condition numbers far below 1/eps of that type (eps = 6e-8
 * for FP32) for the inverses to keep their accuracy.  Errors: FUSE_EINVAL (NULL). */
fuse_status fuse_conditioning(fuse_ctx* ctx, double out[3]);

/* Size in bytes of the resumable ADMM state (Lambda1, U1 = P1 + Lambda1, Lambda2,
 * U2 = P2 + Lambda2, X, Sigma, the adjoint partial sums), in that order; Sigma is stored as
 * Sig'[tau][k][c][m] = Sigma_{tau k}(m + k) over the kept offsets (all of W, or W+ in
 * half-window mode, row-major). */
fuse_status fuse_state_bytes(fuse_ctx* ctx, size_t* bytes);

/* Copy the state to / from a buffer of fuse_state_bytes bytes (host or device; uses
 * cudaMemcpyAsync with cudaMemcpyDefault, synchronous on return).  fuse_set_state makes
 * the next warm fuse_solve continue bit-identically from the saved iteration. */
fuse_status fuse_get_state(fuse_ctx* ctx, void* dst);
fuse_status fuse_set_state(fuse_ctx* ctx, const void* src);

/* Options (FUSE_OPT_*).  Launch options that do not fit the problem return FUSE_EINVAL and
 * leave the previous setting in place. */
fuse_status fuse_set_option(fuse_ctx* ctx, int option, long long value);

/* Current value of an option (FUSE_OPT_*). */
fuse_status fuse_get_option(fuse_ctx* ctx, int option, long long* value);

/* Launch-shape tuner: with the context's weights and the given inputs (as in fuse_solve), times
 * `iters` iterations for each candidate shape of the latent pass (consumer threads 128/192/256,
 * ring slots 4/6/8/12/16/24, bands per block 1/2; shapes that do not fit are skipped) and of the
 * FFT passes (rows per block 1..8, columns per block 2..16) and keeps the fastest.  Results do not depend on the shapes (bit-identical).
 * Leaves the context without state: the next fuse_solve starts from zero.  Synchronous. */
fuse_status fuse_autotune(fuse_ctx* ctx, const void* Yl_dev, const void* Yh_dev, int iters);

/* Wait for all work issued on the context's stream and report device-side failures:
 * FUSE_ETIMEOUT if a bounded barrier wait inside a kernel gave up since the last check
 * (the results of that work are then invalid), FUSE_ECUDA on an execution error. */
fuse_status fuse_sync(fuse_ctx* ctx);

/* Profile counters since the last reset: kernel group `which` (FUSE_K_*): total device time
 * in ms (only with FUSE_OPT_PROFILE, else 0) and launch count.  Synchronises the stream.
 * reset != 0 clears the counters after reading. */
fuse_status fuse_profile(fuse_ctx* ctx, int which, double* ms, long long* launches, int reset);

/* The regulariser value phi(X) = sum_i sum_{tau in W} omega_{i tau} ||P_{i tau}(X)||_1 written
 * to phi_dev[0] (device, one double), without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate device memory and
 * so cannot create a fuse_ctx: a host application that owns a fixed GPU memory budget and
 * hands out every byte itself, or a loop with a latency bound that cannot afford cudaMalloc's
 * implicit device synchronisation.
 *   X_dev      [L_s][H][W] of dtype (FUSE_F32 or FUSE_F64), device
 *   omega_dev  [|W|][H][W] of wdtype (FUSE_F32/FUSE_BF16 with FUSE_F32, FUSE_F64 with FUSE_F64),
 *              as produced by fuse_weights / read by fuse_get_weights
 *   stream     cudaStream_t (as void*), NULL = legacy default stream; asynchronous.
 * Scratch: per-block partial sums in one file-scope device array of 2^18 doubles (2 MiB),
 * held on every GPU that loads the library until the process exits.  The problem must need
 * at most that many partials: ceil(H*W/256) * |W| <= 262144, else FUSE_EUNSUPPORTED (and
 * no work is issued).  Every call shares the array and overwrites the slots it uses before
 * reading them; calls whose execution overlaps on the GPU (different streams, or graphs
 * replayed concurrently) race on it.  The first call on each device looks up the array's
 * device address (once, with that device current); make that first call before any stream
 * capture.  Calls no allocating routine.  Errors: FUSE_EINVAL, FUSE_EUNSUPPORTED, FUSE_ECUDA. */
fuse_status fuse_phi_static(const void* X_dev, const void* omega_dev, int H, int W, int L_s, int K,
                            int S, fuse_dtype dtype, fuse_dtype wdtype, double* phi_dev, void* stream);

/* ---- Reverse pass (differentiation of K unrolled iterations) -----------------------------
 * The ADMM of Sec. IV run for a fixed number K of iterations from zero state is a
 * differentiable map (Y_l, Y_h, lambda1, lambda2, rho, omega) -> X_K, with omega itself a
 * function of the guide (eq. wts); the paper does not differentiate it, these entry points
 * do, by the exact adjoint of every update in reverse order: the soft threshold of eq. Qj_main
 * (derivative taken as 0 at |v| = mu), the closed forms of eqs. Qm_update and Qh_update, the
 * dual updates, and the X update of eq. inv (A is symmetric, so its adjoint is the same
 * per-frequency division).  fuse_grad_backward returns the data-path gradients;
 * fuse_grad_weights the weight and guide gradients.
 *
 * Checkpointing: the forward keeps, for each of its iterations, X and the entering Lambda1,
 * Lambda2 and Sigma (the tape).  With FUSE_OPT_GRAD_SEGMENT = s > 0 the iterations are grouped
 * in segments of s: the tape holds s iterations, the full state entering each later segment is
 * saved, and the reverse pass re-runs each earlier segment from its saved state (recompute).
 * Device memory: fuse_grad_bytes.  The workspace is allocated on first use and kept. */

/* Bytes of the reverse-pass workspace for `iters` iterations under the current options. */
fuse_status fuse_grad_bytes(fuse_ctx* ctx, int iters, size_t* bytes);

/* Forward pass with checkpoints: `iters` iterations from zero state on Y_l, Y_h (as in
 * fuse_solve, cold start) with the context's weights; X of the last iteration to X_out
 * (nullable, device [L_s][H][W]).  Leaves the context's state as fuse_solve would.  Any later
 * call that changes inputs or state (fuse_solve, fuse_weights, fuse_set_weights,
 * fuse_set_state, FUSE_OPT_HALF_WINDOW) invalidates the checkpoints.  Asynchronous.
 * Errors: FUSE_EINVAL, FUSE_ESTATE (no weights), FUSE_EUNSUPPORTED (L_s > 32), FUSE_ENOMEM. */
fuse_status fuse_grad_forward(fuse_ctx* ctx, const void* Yl_dev, const void* Yh_dev, int iters,
                              void* X_out);

/* Reverse pass for the last fuse_grad_forward, for the loss L with
 *   Xbar_dev  dL/dX  of the last iterate, device [L_s][H][W] (nullable),
 *   Zbar_dev  dL/dZ, Z = X E, device [L_l][H][W] (nullable; both given: their effects add).
 * Outputs (each nullable): Yl_bar_dev dL/dY_l [L_l][H/ratio][W/ratio], Yh_bar_dev dL/dY_h
 * [L_h][H][W] (device, dtype), param_bar[3] = dL/dlambda1, dL/dlambda2, dL/drho (host,
 * double; when given the call synchronises the stream).  With one segment the tape is kept
 * and the call may be repeated with other dL/dX; with several segments the recomputation
 * overwrites the context's ADMM state (the next warm fuse_solve starts from zero) and the
 * checkpoints are consumed.  Sums are in the context's dtype, parameter sums in FP64.
 * Errors: FUSE_EINVAL (no dL/dX nor dL/dZ), FUSE_ESTATE (no valid forward),
 * FUSE_ENONFINITE, FUSE_ECUDA. */
fuse_status fuse_grad_backward(fuse_ctx* ctx, const void* Xbar_dev, const void* Zbar_dev,
                               void* Yl_bar_dev, void* Yh_bar_dev, double* param_bar);

/* Weight and guide gradients of the last fuse_grad_backward, which must have run with
 * FUSE_OPT_GRAD_WEIGHTS = 1 (else FUSE_ESTATE).  The weights enter the iterations only through
 * the thresholds mu = lambda2 omega / rho (eq. Qj_main).
 *   omega_bar_dev  nullable, device [|W|][H][W] of dtype: dL/domega for the weight array the
 *                  context holds (fuse_weights / fuse_set_weights layout).  In half-window mode
 *                  the solver reads only the kept offsets, whose weights also threshold their
 *                  mirrors: their entries carry both, and the other offsets' entries are 0.
 *   guide_dev      the guide given to fuse_weights, device [L_guide][H][W] of dtype (needed
 *                  for guide_bar_dev only)
 *   guide_bar_dev  nullable, device [L_guide][H][W] of dtype: dL/dguide through eq. wts,
 *                  dL/dG = sum_tau sum_k D_{tau k}^T (-2/h^2 omega_bar omega D_{tau k} G).
 *                  When the guide is Y_h, the full dL/dY_h is this plus fuse_grad_backward's
 *                  Yh_bar (the data path).
 * Asynchronous.  Errors: FUSE_ESTATE, FUSE_EINVAL (guide_bar without guide), FUSE_ENOMEM. */
fuse_status fuse_grad_weights(fuse_ctx* ctx, void* omega_bar_dev, const void* guide_dev,
                              void* guide_bar_dev);

/* fuse_grad_forward followed by fuse_grad_backward. */
fuse_status fuse_grad(fuse_ctx* ctx, const void* Yl_dev, const void* Yh_dev, int iters,
                      const void* Xbar_dev, const void* Zbar_dev, void* X_out, void* Yl_bar_dev,
                      void* Yh_bar_dev, double* param_bar);

/* Device self-check.  which = 1: a kernel waits (bounded) on a barrier that nothing completes;
 * returns FUSE_OK when the wait gave up and its timeout was reported to the host as designed,
 * leaving the context usable.  Synchronous. */
fuse_status fuse_selftest(fuse_ctx* ctx, int which);

/* ---- Batches of independent problems (uneven sizes) ------------------------------------
 * A batch runs the ADMM of several contexts together: each iteration is one launch per
 * phase (right-hand side, three FFT passes, B X, pixel updates, latent pass) over the work of
 * every problem, and the whole iteration loop is replayed from captured CUDA graphs as in
 * FUSE_OPT_GRAPH.  The contexts must share dtype,
 * wdtype, K, S, L_s (<= 32), blur size and half-window mode; sizes (H, W, ratio, L_l, L_h) may
 * differ.  The batch does not own the contexts: destroy the batch before them.  Creating a
 * batch moves every context onto the batch's stream. */
typedef struct fuse_batch fuse_batch;

/* Build the launch tables for ctxs[0..n) (device memory for the tables is allocated here).
 * Errors: FUSE_EINVAL (mismatched or duplicate contexts), FUSE_EUNSUPPORTED, FUSE_ENOMEM. */
fuse_status fuse_batch_create(fuse_batch** out, fuse_ctx* const* ctxs, int n, void* stream);

/* Solve every problem of the batch from a zero start for `iters` iterations.  Yl[i], Yh[i] are
 * the device inputs of problem i (as in fuse_solve); X_out, Z_out are nullable arrays of
 * nullable device outputs.  Every context must hold weights (fuse_weights or
 * fuse_set_weights).  Asynchronous on the batch's stream. */
fuse_status fuse_batch_solve(fuse_batch* b, const void* const* Yl, const void* const* Yh, int iters,
                             void* const* X_out, void* const* Z_out);

/* End-to-end batch call on HOST buffers (the batch counterpart of fuse_run_host): for every
 * problem i, copies Yl_host[i] [L_l][H/ratio][W/ratio] and Yh_host[i] [L_h][H][W] (and
 * guide_host[i] [L_guide][H][W] when guide_host and guide_host[i] are non-NULL; otherwise the
 * guide is Y_h) to device staging buffers, computes problem i's weights (eq. wts), solves all
 * problems together from a zero start for `iters` iterations (fuse_batch_solve) and copies
 * X_host[i] [L_s][H][W] and/or Z_host[i] [L_l][H][W] back (X_host, Z_host and their entries
 * nullable).  Element type of every buffer: the contexts' dtype; host buffers should be pinned
 * for asynchronous copies.  The staging buffers are allocated on first use and kept by each
 * context.  Synchronous: returns after the results are in host memory and the device-side
 * checks of fuse_batch_sync.  Errors: FUSE_EINVAL (NULL inputs, guide NULL with
 * L_guide != L_h, iters < 0), FUSE_ESTATE, FUSE_ENOMEM, FUSE_ECUDA, FUSE_ETIMEOUT. */
fuse_status fuse_batch_run_host(fuse_batch* b, const void* const* Yl_host, const void* const* Yh_host,
                                const void* const* guide_host, int iters, void* const* X_host,
                                void* const* Z_host);

/* FUSE_OPT_PROFILE, FUSE_OPT_GRAPH, FUSE_OPT_LATENT_THREADS, FUSE_OPT_LATENT_STAGES,
 * FUSE_OPT_LATENT_BANDS. */
fuse_status fuse_batch_set_option(fuse_batch* b, int option, long long value);

/* Current value of a batch option (the options of fuse_batch_set_option).  Errors: FUSE_EINVAL. */
fuse_status fuse_batch_get_option(fuse_batch* b, int option, long long* value);

/* Launch-shape tuner of a batch (latent pass: consumer threads 128/160/192/256, ring slots
 * 6/8/12/16, bands per block 1/2/4/8; shapes that do not fit are skipped),
 * timing `iters` batched iterations per candidate; inputs as in fuse_batch_solve.  Synchronous. */
fuse_status fuse_batch_autotune(fuse_batch* b, const void* const* Yl, const void* const* Yh, int iters);

/* As fuse_profile, for the batched launches (FUSE_K_LATENT: the batched latent pass). */
fuse_status fuse_batch_profile(fuse_batch* b, int which, double* ms, long long* launches, int reset);

/* Synchronise the batch's stream and report device-side failures of any of its problems. */
fuse_status fuse_batch_sync(fuse_batch* b);

fuse_status fuse_batch_destroy(fuse_batch* b);
const char* fuse_batch_last_error(const fuse_batch* b);

/* Last error text of the context ("" if none); valid until the next call on ctx. */
const char* fuse_last_error(const fuse_ctx* ctx);

/* Clear the sticky error of the context. */
fuse_status fuse_reset_error(fuse_ctx* ctx);

/* Static name of a status code. */
const char* fuse_status_string(fuse_status s);

#ifdef __cplusplus
}
#endif

#endif /* FUSE_H */
