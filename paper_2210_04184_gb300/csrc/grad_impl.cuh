// Host side of the reverse pass through K unrolled ADMM iterations (Sec. IV run for a fixed
// number of iterations from zero state, differentiated).  Included by fuse_api.cu after the
// forward launch sequence; the device kernels are in k_grad.cuh.
//
// Forward with checkpoints: iterations are grouped in segments of `seg` iterations.  While
// the forward runs, the state entering the first iteration of every segment but the first is
// saved whole (Lambda1, U1, Lambda2, U2, Sigma, planes), and every iteration's X and its
// entering Lambda1, Lambda2 and Sigma go to a tape of `seg` slots.  The reverse pass walks the
// segments backwards; for each but the last it restores the segment's checkpoint and re-runs the
// segment's iterations to refill the tape (recomputation), then reverses them.
#pragma once

struct GradWork {
    int iters = 0, seg = 0, nseg = 0;
    int cap_seg = 0, cap_ck = 0;
    size_t sig_bytes = 0;
    long long epoch = -1;
    // tape: [cap_seg] slots of X, Lambda1, Lambda2 (images) and Sigma entering the iteration
    void *tX = nullptr, *tL1 = nullptr, *tL2 = nullptr, *tSig = nullptr;
    // checkpoints: [cap_ck] blocks of Lambda1, U1, Lambda2, U2, Sigma, planes
    void* ck = nullptr;
    size_t ck_bytes = 0;
    // reverse-pass buffers
    void *Sb = nullptr, *planesB = nullptr, *Xb = nullptr, *Cb = nullptr, *U1b = nullptr, *L1b = nullptr;
    void *L2b = nullptr, *BXt = nullptr, *BXb = nullptr, *Xp = nullptr, *D9ab = nullptr, *D9bb = nullptr;
    void *Krho = nullptr, *Klam = nullptr, *Kmu = nullptr, *MhT = nullptr;
    double *lat_part = nullptr, *px_part = nullptr;
    size_t n_lat_part = 0, n_px_part = 0;
    // launch shape of the bulk-copy latent reverse pass (tma = 0: the register-staged kernel)
    int tma = 0, tb_Ty = 1, tb_ncons = 0, tb_D = 4;
    size_t tb_smem = 0;
    // dL/domega [|W|][H][W] (allocated when FUSE_OPT_GRAD_WEIGHTS is on) and the guide step's
    // box sums; omb_valid: the last reverse pass accumulated omb
    void *omb = nullptr, *Abox = nullptr;
    bool omb_valid = false;
    // the taped forward loop and the reverse loop captured as CUDA graphs, with the launch
    // configuration they were captured for and the launches they hold
    cudaGraphExec_t gfwd = nullptr, gbwd = nullptr;
    std::vector<long long> key_f, key_b;
    long long nl_f = 0, nll_f = 0, nl_b = 0, nll_b = 0;
    std::vector<void*> allocs;
};

namespace {

void grad_free(GradWork* g) {
    if (!g) return;
    if (g->gfwd) cudaGraphExecDestroy(g->gfwd);
    if (g->gbwd) cudaGraphExecDestroy(g->gbwd);
    for (void* p : g->allocs)
        if (p) cudaFree(p);
    g->allocs.clear();
    delete g;
}

fuse_status galloc(fuse_ctx* c, GradWork* g, void** p, size_t bytes) {
    if (c->fault_alloc >= 0 && c->alloc_count++ == c->fault_alloc)
        return fail(c, FUSE_ENOMEM, "injected allocation failure (FUSE_FAULT_ALLOC)");
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail_cuda(c, "cudaMalloc (reverse-pass workspace)", e);
    }
    g->allocs.push_back(*p);
    return FUSE_OK;
}

// Segment length for `iters` iterations under the context's option (0 = one segment).
int grad_segment(const fuse_ctx* c, int iters) {
    if (iters <= 0) return 1;
    return (c->grad_seg <= 0 || c->grad_seg >= iters) ? iters : c->grad_seg;
}

size_t grad_ck_bytes(const fuse_ctx* c) {
    return 4 * c->n * c->Ls * c->esz + c->sig_bytes + c->plane_bytes;
}

// Device bytes of the reverse-pass workspace for `iters` iterations.
size_t grad_bytes(const fuse_ctx* c, int iters) {
    const int seg = grad_segment(c, iters);
    const int nseg = iters > 0 ? (iters + seg - 1) / seg : 1;
    const size_t img = c->n * c->Ls * c->esz;
    const size_t tape = (size_t)seg * (3 * img + c->sig_bytes);
    const size_t ck = (size_t)(nseg - 1) * grad_ck_bytes(c);
    const size_t bufs = c->sig_bytes + c->plane_bytes + 10 * img + c->nl * c->Ls * c->esz;
    return tape + ck + bufs;
}

template <typename T>
void upload_mat(std::vector<T>& h, const std::vector<double>& v) {
    h.resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) h[i] = (T)v[i];
}

// (Re)allocates the workspace for `iters` iterations.
fuse_status grad_prepare(fuse_ctx* c, int iters) {
    const int seg = grad_segment(c, iters);
    const int nseg = iters > 0 ? (iters + seg - 1) / seg : 1;
    GradWork* g = c->gw;
    if (g && (g->cap_seg < seg || g->cap_ck < nseg - 1 || g->sig_bytes != c->sig_bytes)) {
        CK(c, cudaStreamSynchronize(c->stream));
        grad_free(g);
        c->gw = g = nullptr;
    }
    if (!g) {
        g = new (std::nothrow) GradWork();
        if (!g) return fail(c, FUSE_ENOMEM, "host allocation of the reverse-pass workspace");
        c->gw = g;
        const size_t img = c->n * c->Ls * c->esz;
        g->cap_seg = seg;
        g->cap_ck = nseg - 1;
        g->sig_bytes = c->sig_bytes;
        g->ck_bytes = grad_ck_bytes(c);
        fuse_status st = FUSE_OK;
        auto A = [&](void** p, size_t b) { if (st == FUSE_OK) st = galloc(c, g, p, b); };
        A(&g->tX, (size_t)seg * img);
        A(&g->tL1, (size_t)seg * img);
        A(&g->tL2, (size_t)seg * img);
        A(&g->tSig, (size_t)seg * c->sig_bytes);
        A(&g->ck, (size_t)g->cap_ck * g->ck_bytes);
        A(&g->Sb, c->sig_bytes);
        A(&g->planesB, c->plane_bytes);
        void** imgs[] = {&g->Xb, &g->Cb, &g->U1b, &g->L1b, &g->L2b, &g->BXt, &g->BXb, &g->Xp, &g->D9bb};
        for (void** p : imgs) A(p, img);
        A(&g->D9ab, c->nl * c->Ls * c->esz);
        // constant matrices of the parameter derivatives
        const int Ls = c->Ls, Lh = c->Lh;
        std::vector<double> GG((size_t)Ls * Ls), FGGF((size_t)Ls * Ls), Kr(GG.size()), Kl(GG.size()),
            Km(GG.size()), MhT((size_t)Ls * Lh);
        for (int i = 0; i < Ls; ++i)
            for (int j = 0; j < Ls; ++j) {
                double s = 0;
                for (int k = 0; k < Lh; ++k) s += c->hER[(size_t)i * Lh + k] * c->hER[(size_t)j * Lh + k];
                GG[(size_t)i * Ls + j] = s;
            }
        std::vector<double> tmp((size_t)Ls * Ls);
        for (int i = 0; i < Ls; ++i)
            for (int j = 0; j < Ls; ++j) {
                double s = 0, m = 0;
                for (int k = 0; k < Ls; ++k) {
                    s += c->hF[(size_t)i * Ls + k] * GG[(size_t)k * Ls + j];
                    m += c->hM1[(size_t)i * Ls + k] * c->hM1[(size_t)k * Ls + j];
                }
                tmp[(size_t)i * Ls + j] = s;
                Km[(size_t)i * Ls + j] = -m;                      // d M1 / d rho = -M1 M1
            }
        for (int i = 0; i < Ls; ++i)
            for (int j = 0; j < Ls; ++j) {
                double s = 0;
                for (int k = 0; k < Ls; ++k) s += tmp[(size_t)i * Ls + k] * c->hF[(size_t)k * Ls + j];
                FGGF[(size_t)i * Ls + j] = s;
            }
        // F = (I + lambda1/rho G G^T)^{-1}: dF/drho = lambda1/rho^2 F GG^T F, dF/dlambda1 = -1/rho F GG^T F
        for (size_t q = 0; q < FGGF.size(); ++q) {
            Kr[q] = c->lam1 / (c->rho * c->rho) * FGGF[q];
            Kl[q] = -FGGF[q] / c->rho;
        }
        // D9b = Y_h Mh with Mh = lambda1/rho R^T E^T  =>  Y_h bar = D9b bar Mh^T
        for (int i = 0; i < Ls; ++i)
            for (int k = 0; k < Lh; ++k) MhT[(size_t)i * Lh + k] = c->lam1 / c->rho * c->hER[(size_t)i * Lh + k];
        auto U = [&](void** p, const std::vector<double>& v) {
            if (st != FUSE_OK) return;
            const size_t bytes = v.size() * c->esz;
            st = galloc(c, g, p, bytes);
            if (st != FUSE_OK) return;
            cudaError_t e;
            if (c->dtype == FUSE_F64) {
                e = cudaMemcpy(*p, v.data(), bytes, cudaMemcpyHostToDevice);
            } else {
                std::vector<float> h;
                upload_mat(h, v);
                e = cudaMemcpy(*p, h.data(), bytes, cudaMemcpyHostToDevice);
            }
            if (e != cudaSuccess) st = fail_cuda(c, "cudaMemcpy (reverse-pass constants)", e);
        };
        U(&g->Krho, Kr);
        U(&g->Klam, Kl);
        U(&g->Kmu, Km);
        U(&g->MhT, MhT);
        // launch shape of the bulk-copy latent reverse pass: about 128 consumer threads of 16 bytes
        // of pixels each over full rows, a ring of 4 slots of two planes (taped state, adjoint)
        {
            const int vec = (int)(16 / c->esz), tpr = c->W / vec;
            int Ty = 128 / tpr;
            Ty = Ty < 1 ? 1 : (Ty > c->H ? c->H : Ty);
            while (Ty > 1 && ((tpr * Ty + 31) / 32) * 32 + 32 > 288) --Ty;
            const int ncons = ((tpr * Ty + 31) / 32) * 32;
            const size_t smem = (size_t)g->tb_D * 2 * Ty * c->W * c->esz + (size_t)(2 * c->S + 1) * Ty * c->W * c->esz +
                                2 * (size_t)g->tb_D * 8;
            g->tma = (c->lat_impl == 1 && ncons + 32 <= 288 && smem <= (size_t)kMaxSmem) ? 1 : 0;
            g->tb_Ty = Ty;
            g->tb_ncons = ncons;
            g->tb_smem = smem;
        }
        // partial sums: one slot per block of the latent and pixel reverse kernels
        const unsigned rowsW = (unsigned)(c->half ? c->S + 1 : 2 * c->S + 1);
        const int lty = g->tma ? g->tb_Ty : c->lat_Ty;
        g->n_lat_part = (size_t)((c->H + lty - 1) / lty) * c->Ls * rowsW;
        g->n_px_part = 3 * ((c->n + 127) / 128);
        A((void**)&g->lat_part, g->n_lat_part * sizeof(double));
        A((void**)&g->px_part, g->n_px_part * sizeof(double));
        if (st != FUSE_OK) {
            grad_free(g);
            c->gw = nullptr;
            return st;
        }
    }
    g->iters = iters;
    g->seg = seg;
    g->nseg = nseg;
    return FUSE_OK;
}

template <typename T>
struct GradImpl {
    static constexpr int VEC = 16 / sizeof(T);

    static fuse_status set_attrs(fuse_ctx* c) {
        cudaError_t e;
        if constexpr (sizeof(T) == 8) {
            e = latent_bwd_set_smem<T, double>(c->K, kMaxSmem);
        } else {
            e = latent_bwd_set_smem<T, float>(c->K, kMaxSmem);
            if (e == cudaSuccess) e = latent_bwd_set_smem<T, __nv_bfloat16>(c->K, kMaxSmem);
        }
        CK(c, e);
        return FUSE_OK;
    }

    // out = A^{-1} in (eq. inv), the forward's three FFT launches on other buffers.
    static fuse_status solve_A(fuse_ctx* c, cudaStream_t s, const void* in, void* out) {
        const FFTArgs<T> fa{(const T*)in, (cplx<T>*)c->Y, (T*)out, (const T*)c->fpf, c->H, c->W, c->Ls,
                            c->planW, c->planH, (const cplx<T>*)c->twW, (const cplx<T>*)c->twH, c->fr_rpb, c->fc_cw,
                            c->fft_impl == 1 ? (const T*)c->fT : nullptr};
        const fuse_status st = Impl<T>::dft_solve(c, s, fa);
        if (st != FUSE_OK) return st;
        c->launches_all += 3;
        return FUSE_OK;
    }

    // MODE 0: out = B in; MODE 1: out = B^T in + U2 + (adjoint sum of planes).
    template <int MODE>
    static fuse_status stencil(fuse_ctx* c, cudaStream_t s, const void* in, void* out, const void* taps,
                               const void* U2, const void* planes) {
        const StencilArgs<T> a{(const T*)in, (T*)out, (const T*)taps, c->bw, c->H, c->W,
                               (const T*)U2, (const T*)planes, c->S, c->half};
        Impl<T>::template stencil_launch<MODE>(c, s, a);
        c->launches_all++;
        CKL(c, "stencil_kernel (reverse pass)");
        return FUSE_OK;
    }

    template <typename WT>
    static void latent_bwd(fuse_ctx* c, cudaStream_t s, const void* Xt, const void* Sin) {
        GradWork* g = c->gw;
        const unsigned rowsW = (unsigned)(c->half ? c->S + 1 : 2 * c->S + 1);
        if (g->tma) {
            dim3 grid((unsigned)((c->H + g->tb_Ty - 1) / g->tb_Ty), (unsigned)c->Ls, rowsW);
            const LatentBwdArgs<T, WT> a{(const T*)Xt, (const WT*)c->omega, (const T*)Sin, (T*)g->Sb, (const T*)g->Cb,
                                         (T*)g->planesB, g->lat_part, c->H, c->W, c->Ls, c->S, g->tb_Ty,
                                         g->tb_ncons, g->tb_D, (T)(c->lam2 / c->rho), c->d_err, c->wait_limit,
                                         c->half};
            latent_bwd_tma_launch<T, WT>(a, c->K, grid, (unsigned)(g->tb_ncons + 32), g->tb_smem, s);
            return;
        }
        dim3 grid((unsigned)((c->H + c->lat_Ty - 1) / c->lat_Ty), (unsigned)c->Ls, rowsW);
        latent_bwd_reg_launch<T, WT>((const T*)Xt, (const WT*)c->omega, (const T*)Sin, (T*)g->Sb, (const T*)g->Cb,
                                     (T*)g->planesB, g->lat_part, c->H, c->W, c->Ls, c->S, c->lat_Ty,
                                     (T)(c->lam2 / c->rho), c->half, c->K, grid,
                                     (unsigned)((c->lat_threads + 31) / 32 * 32), c->lat_smem, s);
    }

    template <typename WT>
    static void omega_bwd(fuse_ctx* c, cudaStream_t s, const void* Xt, const void* Sin) {
        GradWork* g = c->gw;
        const unsigned kept = (unsigned)(c->half ? c->nW / 2 : c->nW);
        dim3 grid((unsigned)((c->n + 255) / 256), kept);
        const T coef = (T)(c->lam2 / c->rho);
        const T scale = (T)((c->half ? 2.0 : 1.0) * c->lam2 / c->rho);
        omega_bwd_launch<T, WT>((const T*)Xt, (const WT*)c->omega, (const T*)Sin, (const T*)g->Sb, (const T*)g->Cb,
                                (T*)g->omb, c->H, c->W, c->Ls, c->S, coef, scale, c->half, c->K, grid, s);
    }

    static fuse_status omega_bwd_any(fuse_ctx* c, cudaStream_t s, const void* Xt, const void* Sin) {
        if constexpr (sizeof(T) == 8) {
            omega_bwd<double>(c, s, Xt, Sin);
        } else {
            if (c->wdtype == FUSE_BF16) omega_bwd<__nv_bfloat16>(c, s, Xt, Sin);
            else omega_bwd<float>(c, s, Xt, Sin);
        }
        c->launches_all++;
        CKL(c, "omega_bwd_kernel");
        return FUSE_OK;
    }

    static fuse_status latent_bwd_any(fuse_ctx* c, cudaStream_t s, const void* Xt, const void* Sin) {
        if constexpr (sizeof(T) == 8) {
            latent_bwd<double>(c, s, Xt, Sin);
        } else {
            if (c->wdtype == FUSE_BF16) latent_bwd<__nv_bfloat16>(c, s, Xt, Sin);
            else latent_bwd<float>(c, s, Xt, Sin);
        }
        c->launches_all++;
        CKL(c, "latent_bwd_kernel");
        return FUSE_OK;
    }

    static fuse_status pixel_bwd(fuse_ctx* c, cudaStream_t s, const void* Xt, const void* L1t, const void* L2t) {
        GradWork* g = c->gw;
        const PixelBwdArgs<T> a{(const T*)Xt, (const T*)g->BXt, (const T*)L1t, (const T*)L2t,
                                (const T*)g->U1b, (const T*)g->Cb, (T*)g->L1b, (T*)g->L2b, (T*)g->Xp, (T*)g->BXb,
                                (T*)g->D9ab, (T*)g->D9bb, (const T*)c->D9a, (const T*)c->D9b, (const T*)c->M1,
                                (const T*)c->F, (const T*)g->Krho, (const T*)g->Klam, (const T*)g->Kmu,
                                g->px_part, c->H, c->W, c->Ls, c->d, (T)c->rho, (const uint8_t*)c->mask};
        const unsigned blocks = (unsigned)((c->n + 127) / 128);
        pixel_bwd_launch<T>(a, blocks, s);
        c->launches_all++;
        CKL(c, "pixel_bwd_kernel");
        return FUSE_OK;
    }

    // Reverse of iteration t (tape slot `slot`), `last` = the final iteration, whose outputs
    // other than X have zero adjoints; on entry Xb holds dL/dX_t for the last iteration.
    static fuse_status reverse_step(fuse_ctx* c, cudaStream_t s, int t, int slot, bool last) {
        GradWork* g = c->gw;
        const size_t img = c->n * c->Ls * c->esz;
        const char* Xt = (const char*)g->tX + (size_t)slot * img;
        fuse_status st;
        if (!last) {
            // X_0 = 0 and Sigma_0 = 0, so the first latent pass has v = 0 and no threshold term
            if (t > 0) {
                const char* Sin = (const char*)g->tSig + (size_t)slot * c->sig_bytes;
                if (c->grad_weights) {
                    st = omega_bwd_any(c, s, Xt, Sin);          // reads Sigmabar' before it is overwritten
                    if (st != FUSE_OK) return st;
                }
                st = latent_bwd_any(c, s, Xt, Sin);
                if (st != FUSE_OK) return st;
            }
            st = stencil<0>(c, s, Xt, g->BXt, c->tapsB, nullptr, nullptr);
            if (st != FUSE_OK) return st;
            st = pixel_bwd(c, s, Xt, (const char*)g->tL1 + (size_t)slot * img, (const char*)g->tL2 + (size_t)slot * img);
            if (st != FUSE_OK) return st;
            if (t == 0) return FUSE_OK;                       // X_0 = A^{-1} 0 does not depend on anything
            // Xbar = B^T BXbar + Xp + sum D^T vbar
            st = stencil<1>(c, s, g->BXb, g->Xb, c->tapsT, g->Xp, g->planesB);
            if (st != FUSE_OK) return st;
        } else if (t == 0) {
            return FUSE_OK;
        }
        st = solve_A(c, s, g->Xb, g->Cb);
        if (st != FUSE_OK) return st;
        return stencil<0>(c, s, g->Cb, g->U1b, c->tapsB, nullptr, nullptr);
    }
};

// One directly launched forward iteration in tape slot `slot` of a segment of `len` iterations.
// The entering Lambda1, Lambda2 are copied to the slot and X after the iteration; the latent
// pass reads Sigma from the slot and writes the next slot (the context's state after the
// segment's last iteration), so taping Sigma costs no extra pass over it.
fuse_status taped_iteration(fuse_ctx* c, int slot, int len) {
    GradWork* g = c->gw;
    const size_t img = c->n * c->Ls * c->esz;
    CK(c, cudaMemcpyAsync((char*)g->tL1 + (size_t)slot * img, c->Lam1, img, cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync((char*)g->tL2 + (size_t)slot * img, c->Lam2, img, cudaMemcpyDeviceToDevice, c->stream));
    c->lat_in = (char*)g->tSig + (size_t)slot * c->sig_bytes;
    c->lat_out = slot + 1 < len ? (char*)g->tSig + (size_t)(slot + 1) * c->sig_bytes : c->Sig;
    fuse_status st = c->dtype == FUSE_F64 ? Impl<double>::iterate(c, c->stream, false)
                                          : Impl<float>::iterate(c, c->stream, false);
    c->lat_in = c->lat_out = nullptr;
    if (st != FUSE_OK) return st;
    c->launches_all += 7;
    c->launches_latent += 1;
    CK(c, cudaMemcpyAsync((char*)g->tX + (size_t)slot * img, c->X, img, cudaMemcpyDeviceToDevice, c->stream));
    return FUSE_OK;
}

fuse_status checkpoint_copy(fuse_ctx* c, int j, bool save) {
    GradWork* g = c->gw;
    const size_t img = c->n * c->Ls * c->esz;
    char* p = (char*)g->ck + (size_t)(j - 1) * g->ck_bytes;
    void* bufs[] = {c->Lam1, c->U1, c->Lam2, c->U2, c->Sig, c->planes};
    const size_t sz[] = {img, img, img, img, c->sig_bytes, c->plane_bytes};
    for (int q = 0; q < 6; ++q) {
        if (save) CK(c, cudaMemcpyAsync(p, bufs[q], sz[q], cudaMemcpyDeviceToDevice, c->stream));
        else CK(c, cudaMemcpyAsync(bufs[q], p, sz[q], cudaMemcpyDeviceToDevice, c->stream));
        p += sz[q];
    }
    return FUSE_OK;
}

// Runs segment j from the context's current state (which must be the state entering it),
// filling the tape; `save` also stores that state as the segment's checkpoint.
fuse_status run_segment(fuse_ctx* c, int j, bool save) {
    GradWork* g = c->gw;
    const int s0 = j * g->seg;
    const int len = std::min(g->seg, g->iters - s0);
    fuse_status st;
    if (save && j > 0) {
        st = checkpoint_copy(c, j, true);
        if (st != FUSE_OK) return st;
    }
    if (j == 0) CK(c, cudaMemsetAsync(g->tSig, 0, c->sig_bytes, c->stream));
    else CK(c, cudaMemcpyAsync(g->tSig, c->Sig, c->sig_bytes, cudaMemcpyDeviceToDevice, c->stream));
    for (int k = 0; k < len; ++k) {
        st = taped_iteration(c, k, len);
        if (st != FUSE_OK) return st;
    }
    return FUSE_OK;
}

// Everything a captured loop's launches depend on besides the workspace itself.
std::vector<long long> launch_key(const fuse_ctx* c, int extra) {
    const GradWork* g = c->gw;
    return {g->iters, g->seg, g->nseg, c->lat_impl, c->lat_target, c->lat_stages, c->lat_bpb, c->lt_Ty,
            c->lt_ncons, (long long)c->lt_smem, c->fr_rpb, c->fc_cw, c->half, c->sfmt, (long long)(uintptr_t)c->mask,
            (long long)(uintptr_t)c->Sig, c->grad_weights, (long long)c->wait_limit, extra};
}

// Runs body(stream) on the context stream: directly (profiling, or graphs switched off), else by
// replaying a CUDA graph captured from it, recaptured when the launch configuration changed.
template <typename F>
fuse_status run_captured(fuse_ctx* c, cudaGraphExec_t* exec, std::vector<long long>* key, long long* nl,
                         long long* nll, const std::vector<long long>& want, F&& body) {
    if (c->profile || !c->use_graph) {
        if (*exec) { cudaGraphExecDestroy(*exec); *exec = nullptr; }
        return body(c->stream);
    }
    if (!*exec || *key != want) {
        if (*exec) { cudaGraphExecDestroy(*exec); *exec = nullptr; }
        const long long l0 = c->launches_all, ll0 = c->launches_latent;
        cudaStream_t saved = c->stream;
        CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        c->stream = c->cap_stream;
        fuse_status st = body(c->cap_stream);
        c->stream = saved;
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &gr);
        *nl = c->launches_all - l0;
        *nll = c->launches_latent - ll0;
        c->launches_all = l0;
        c->launches_latent = ll0;
        if (st != FUSE_OK) { if (gr) cudaGraphDestroy(gr); return st; }
        if (e != cudaSuccess) return fail_cuda(c, "cudaStreamEndCapture (reverse pass)", e);
        e = cudaGraphInstantiate(exec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) { *exec = nullptr; return fail_cuda(c, "cudaGraphInstantiate (reverse pass)", e); }
        *key = want;
    }
    CK(c, cudaGraphLaunch(*exec, c->stream));
    c->launches_all += *nl;
    c->launches_latent += *nll;
    return FUSE_OK;
}

fuse_status grad_forward_impl(fuse_ctx* c, const void* Yl, const void* Yh, int iters, void* Xo) {
    fuse_status st = grad_prepare(c, iters);
    if (st != FUSE_OK) return st;
    // D9a, D9b and zero state, as a cold solve
    st = solve_impl(c, Yl, Yh, 0, 0, nullptr, nullptr);
    if (st != FUSE_OK) return st;
    GradWork* g = c->gw;
    if (iters > 0) {
        st = run_captured(c, &g->gfwd, &g->key_f, &g->nl_f, &g->nll_f, launch_key(c, 0), [&](cudaStream_t) {
            for (int j = 0; j < g->nseg; ++j) {
                fuse_status s2 = run_segment(c, j, true);
                if (s2 != FUSE_OK) return s2;
            }
            return FUSE_OK;
        });
        if (st != FUSE_OK) return st;
    }
    c->have_x = true;
    const size_t img = c->n * c->Ls * c->esz;
    if (Xo) CK(c, cudaMemcpyAsync(Xo, c->X, img, cudaMemcpyDeviceToDevice, c->stream));
    g->epoch = ++c->epoch;
    return FUSE_OK;
}

template <typename T>
fuse_status grad_backward_t(fuse_ctx* c, const void* Xbar, const void* Zbar, void* Ylb, void* Yhb, double* pbar) {
    GradWork* g = c->gw;
    cudaStream_t s = c->stream;
    const size_t img = c->n * c->Ls * c->esz;
    fuse_status st = GradImpl<T>::set_attrs(c);
    if (st != FUSE_OK) return st;
    CK(c, cudaMemsetAsync(g->D9ab, 0, c->nl * c->Ls * c->esz, s));
    CK(c, cudaMemsetAsync(g->D9bb, 0, img, s));
    CK(c, cudaMemsetAsync(g->lat_part, 0, g->n_lat_part * sizeof(double), s));
    CK(c, cudaMemsetAsync(g->px_part, 0, g->n_px_part * sizeof(double), s));
    CK(c, cudaMemsetAsync(g->Sb, 0, c->sig_bytes, s));
    CK(c, cudaMemsetAsync(g->L1b, 0, img, s));
    CK(c, cudaMemsetAsync(g->L2b, 0, img, s));
    g->omb_valid = false;
    if (c->grad_weights) {
        if (!g->omb) {
            st = galloc(c, g, &g->omb, (size_t)c->nW * c->n * c->esz);
            if (st != FUSE_OK) return st;
        }
        CK(c, cudaMemsetAsync(g->omb, 0, (size_t)c->nW * c->n * c->esz, s));
    }
    // dL/dX of the last iteration: Xbar + Zbar E^T (Z = X E)
    if (Zbar) {
        st = Impl<T>::band_mix(c, s, Zbar, g->Xb, c->Et, c->n, c->Ll, c->Ls);
        if (st != FUSE_OK) return st;
        if (Xbar) {
            axpy_kernel<T><<<(unsigned)std::min<size_t>((c->n * c->Ls + 255) / 256, 4096), 256, 0, s>>>(
                (T*)g->Xb, (const T*)Xbar, c->n * c->Ls);
            c->launches_all++;
            CKL(c, "axpy_kernel");
        }
    } else {
        CK(c, cudaMemcpyAsync(g->Xb, Xbar, img, cudaMemcpyDeviceToDevice, s));
    }
    const int iters = g->iters;
    const bool recomputed = g->nseg > 1;
    st = run_captured(c, &g->gbwd, &g->key_b, &g->nl_b, &g->nll_b, launch_key(c, 1), [&](cudaStream_t ls) {
        for (int j = g->nseg - 1; j >= 0; --j) {
            const int s0 = j * g->seg;
            const int e0 = std::min(iters, s0 + g->seg);
            fuse_status s2;
            if (j != g->nseg - 1) {
                // refill the tape: restore the segment's entering state and re-run it
                s2 = j == 0 ? zero_state(c, ls) : checkpoint_copy(c, j, false);
                if (s2 != FUSE_OK) return s2;
                s2 = run_segment(c, j, false);
                if (s2 != FUSE_OK) return s2;
            }
            for (int t = e0 - 1; t >= s0; --t) {
                s2 = GradImpl<T>::reverse_step(c, ls, t, t - s0, t == iters - 1);
                if (s2 != FUSE_OK) return s2;
            }
        }
        return FUSE_OK;
    });
    if (st != FUSE_OK) return st;
    g->omb_valid = c->grad_weights != 0;
    if (recomputed) {
        // the context's state is now that of an earlier iteration
        c->have_state = false;
        c->have_x = false;
        g->epoch = -1;
        ++c->epoch;
    }
    if (Ylb) {
        st = Impl<T>::band_mix(c, s, g->D9ab, Ylb, c->Emix, c->nl, c->Ls, c->Ll);
        if (st != FUSE_OK) return st;
    }
    if (Yhb) {
        st = Impl<T>::band_mix(c, s, g->D9bb, Yhb, g->MhT, c->n, c->Ls, c->Lh);
        if (st != FUSE_OK) return st;
    }
    if (pbar) {
        std::vector<double> hl(g->n_lat_part), hp(g->n_px_part);
        CK(c, cudaMemcpyAsync(hl.data(), g->lat_part, hl.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(c, cudaMemcpyAsync(hp.data(), g->px_part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
        double smu = 0, q0 = 0, q1 = 0, q2 = 0;
        for (double v : hl) smu += v;
        for (size_t b = 0; b < hp.size(); b += 3) { q0 += hp[b]; q1 += hp[b + 1]; q2 += hp[b + 2]; }
        // mu = lambda2 omega / rho; D9b = lambda1/rho Y_h R^T E^T
        pbar[0] = q1 + q2 / c->lam1;
        pbar[1] = smu / c->rho;
        pbar[2] = q0 - c->lam2 * smu / (c->rho * c->rho) - q2 / c->rho;
        for (int q = 0; q < 3; ++q)
            if (!std::isfinite(pbar[q])) return fail(c, FUSE_ENONFINITE, "parameter gradient is not finite");
    }
    return FUSE_OK;
}

fuse_status grad_backward_impl(fuse_ctx* c, const void* Xbar, const void* Zbar, void* Ylb, void* Yhb, double* pbar) {
    GradWork* g = c->gw;
    if (!g || g->epoch != c->epoch) return fail(c, FUSE_ESTATE, "no forward pass with checkpoints to reverse");
    if (g->iters <= 1) {
        // X_0 = 0 for every input: all gradients vanish
        if (Ylb) CK(c, cudaMemsetAsync(Ylb, 0, c->nl * c->Ll * c->esz, c->stream));
        if (Yhb) CK(c, cudaMemsetAsync(Yhb, 0, c->n * c->Lh * c->esz, c->stream));
        if (pbar) pbar[0] = pbar[1] = pbar[2] = 0.0;
        g->omb_valid = false;
        if (c->grad_weights) {
            if (!g->omb) {
                fuse_status st = galloc(c, g, &g->omb, (size_t)c->nW * c->n * c->esz);
                if (st != FUSE_OK) return st;
            }
            CK(c, cudaMemsetAsync(g->omb, 0, (size_t)c->nW * c->n * c->esz, c->stream));
            g->omb_valid = true;
        }
        return FUSE_OK;
    }
    return c->dtype == FUSE_F64 ? grad_backward_t<double>(c, Xbar, Zbar, Ylb, Yhb, pbar)
                                : grad_backward_t<float>(c, Xbar, Zbar, Ylb, Yhb, pbar);
}

template <typename T>
fuse_status guide_grad_t(fuse_ctx* c, const void* G, void* Gb) {
    GradWork* g = c->gw;
    cudaStream_t s = c->stream;
    if (!g->Abox) {
        fuse_status st = galloc(c, g, &g->Abox, (size_t)c->nW * c->n * c->esz);
        if (st != FUSE_OK) return st;
    }
    const unsigned nb = (unsigned)((c->n + 255) / 256);
    const T c2 = (T)(-2.0 / (c->h * c->h));
    if constexpr (sizeof(T) == 8) {
        guide_box_kernel<T, double><<<dim3(nb, (unsigned)c->nW), 256, 0, s>>>(
            (const T*)g->omb, (const double*)c->omega, (T*)g->Abox, c->H, c->W, c->K, c2);
    } else {
        if (c->wdtype == FUSE_BF16)
            guide_box_kernel<T, __nv_bfloat16><<<dim3(nb, (unsigned)c->nW), 256, 0, s>>>(
                (const T*)g->omb, (const __nv_bfloat16*)c->omega, (T*)g->Abox, c->H, c->W, c->K, c2);
        else
            guide_box_kernel<T, float><<<dim3(nb, (unsigned)c->nW), 256, 0, s>>>(
                (const T*)g->omb, (const float*)c->omega, (T*)g->Abox, c->H, c->W, c->K, c2);
    }
    CKL(c, "guide_box_kernel");
    guide_bwd_kernel<T><<<dim3(nb, (unsigned)c->Lg), 256, 0, s>>>((const T*)G, (const T*)g->Abox, (T*)Gb, c->H,
                                                                  c->W, c->S);
    CKL(c, "guide_bwd_kernel");
    c->launches_all += 2;
    return FUSE_OK;
}

fuse_status grad_weights_impl(fuse_ctx* c, void* omega_bar, const void* G, void* Gb) {
    GradWork* g = c->gw;
    if (!g || !g->omb_valid) return fail(c, FUSE_ESTATE, "no reverse pass with FUSE_OPT_GRAD_WEIGHTS on");
    if (omega_bar)
        CK(c, cudaMemcpyAsync(omega_bar, g->omb, (size_t)c->nW * c->n * c->esz, cudaMemcpyDeviceToDevice,
                              c->stream));
    if (Gb) {
        if (!G) return fail(c, FUSE_EINVAL, "the guide is needed for its gradient");
        return c->dtype == FUSE_F64 ? guide_grad_t<double>(c, G, Gb) : guide_grad_t<float>(c, G, Gb);
    }
    return FUSE_OK;
}

}  // namespace
