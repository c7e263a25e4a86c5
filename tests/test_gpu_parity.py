"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle, element by element.

Tolerances: FP32 iterates within 1e-5 relative Frobenius error of the FP64 oracle at the same
iteration count; FP64 within 1e-11.  Sizes span several latent row tiles, two 32x32 stencil
tiles and mixed-radix FFT lengths with ragged tails."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300.fuse import (Fusion, FUSE_OPT_GRAPH, FUSE_OPT_LATENT_IMPL,  # noqa: E402
                                         FUSE_OPT_LATENT_STAGES, FUSE_OPT_LATENT_THREADS,
                                         FUSE_OPT_HALF_WINDOW, FUSE_OPT_LATENT_BANDS)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def gpu_solve(p, iters, dtype="f32", wdtype="f32", omega=None, want_state=False, graph=True, opts=()):
    f = Fusion.from_problem(p, dtype=dtype, wdtype=wdtype)
    if not graph:
        f.set_option(FUSE_OPT_GRAPH, 0)
    for o, v in opts:
        f.set_option(o, v)
    td = torch.float64 if dtype == "f64" else torch.float32
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    if omega is None:
        f.weights(yh)
    else:
        f.set_weights(torch.tensor(omega, dtype=f.wtdtype, device="cuda"))
    X, Z = f.solve(yl, yh, iters, want_Z=True)
    f.sync()
    out = dict(X=X.double().cpu().numpy(), Z=Z.double().cpu().numpy(), f=f, yl=yl, yh=yh)
    if want_state:
        out["state"] = f.get_state().cpu().numpy()
    return out


def oracle_solve(p, iters, omega=None):
    om = omega if omega is not None else nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    X, st, su = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S,
                          p.lam1, p.lam2, p.rho, om, iters, fast=True)
    return nlpr.to_lhw(X), st, om


def small(**kw):
    base = dict(H=40, W=40, L_l=6, L_h=2, L_s=3, d=4, blur_size=5, blur_sigma=1.0, K=1, S=2,
                lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=11)
    base.update(kw)
    return synth.make_problem(**base)


# ------------------------------------------------------------------------------ weights


@pytest.mark.parametrize("K,S,H,W", [(1, 2, 40, 40), (2, 3, 36, 64), (0, 1, 24, 20)])
def test_weights_f32_match_oracle(K, S, H, W):
    p = small(K=K, S=S, H=H, W=W)
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    f.weights(torch.tensor(p.Yh, dtype=torch.float32, device="cuda"))
    w = f.get_weights().double().cpu().numpy()
    ref = nlpr.weights(nlpr.to_hwl(p.Yh), K, S, p.h)
    assert w.shape == ref.shape
    assert np.abs(w - ref).max() <= 2e-6


def test_weights_f64_match_oracle():
    p = small(K=2, S=3, H=36, W=64)
    f = Fusion.from_problem(p, dtype="f64", wdtype="f64")
    f.weights(torch.tensor(p.Yh, dtype=torch.float64, device="cuda"))
    w = f.get_weights().cpu().numpy()
    ref = nlpr.weights(nlpr.to_hwl(p.Yh), 2, 3, p.h)
    assert np.abs(w - ref).max() <= 1e-13


def test_weights_bf16_rounding():
    # Both sides round to bf16 (round to nearest even).  The values agree exactly except where
    # the FP32 and FP64 weights straddle a rounding boundary; there they differ by one bf16 step
    # and the FP64 value lies within FP32 error of the midpoint.  exp() scales the FP32 error
    # of the patch distance s/h^2 = -ln(omega) into a relative error of about eps * |ln omega|.
    p = small(K=2, S=3, H=48, W=64)
    f = Fusion.from_problem(p, dtype="f32", wdtype="bf16")
    f.weights(torch.tensor(p.Yh, dtype=torch.float32, device="cuda"))
    w = f.get_weights().double().cpu().numpy()
    ref64 = nlpr.weights(nlpr.to_hwl(p.Yh), 2, 3, p.h)
    ref = nlpr.round_bf16(ref64)
    diff = w != ref
    assert diff.mean() < 1e-3
    if diff.any():
        step = np.abs(w[diff] - ref[diff])
        ulp = np.ldexp(1.0, np.frexp(ref64[diff])[1] - 8)
        assert np.all(step <= ulp * 1.0001)
        mid = (w[diff] + ref[diff]) / 2
        tol = 1e-6 * np.maximum(1.0, np.abs(np.log(mid))) * np.abs(mid)
        assert np.all(np.abs(ref64[diff] - mid) <= tol)


# ------------------------------------------------------------------------------ solve parity


@pytest.mark.parametrize("half", [1, 0])
@pytest.mark.parametrize("iters", [1, 2, 3])
def test_first_iterations_state_parity(iters, half):
    # Element-by-element state after 1, 2, 3 iterations (X update, P1/P2, duals, latent pass).
    # Half-window mode keeps the offsets of W+ = {tau1 > 0} U {tau1 = 0, tau2 > 0} only.
    p = small()
    g = gpu_solve(p, iters, want_state=True, opts=[(FUSE_OPT_HALF_WINDOW, half)])
    Xo, st, _ = oracle_solve(p, iters)
    n = p.H * p.W
    Ls = p.L_s
    s = g["state"].view(np.float32).astype(np.float64)
    img = n * Ls
    lam1, u1, lam2, u2, xs = (s[i * img:(i + 1) * img].reshape(Ls, p.H, p.W) for i in range(5))
    scale = max(np.abs(Xo).max(), 1e-3)
    assert np.abs(g["X"] - Xo).max() <= 2e-6 * max(scale, np.abs(nlpr.to_lhw(st.P2)).max())
    assert np.abs(lam1 - nlpr.to_lhw(st.Lam1)).max() <= 1e-5 * np.abs(nlpr.to_lhw(st.P1)).max()
    assert np.abs(u1 - nlpr.to_lhw(st.P1 + st.Lam1)).max() <= 1e-5 * np.abs(nlpr.to_lhw(st.P1)).max()
    assert np.abs(lam2 - nlpr.to_lhw(st.Lam2)).max() <= 1e-5 * np.abs(nlpr.to_lhw(st.P2)).max()
    assert np.abs(u2 - nlpr.to_lhw(st.P2 + st.Lam2)).max() <= 1e-5 * np.abs(nlpr.to_lhw(st.P2)).max()
    # latent state, stored re-indexed by source pixel: Sig'_{tau k}(m) = Sigma_{tau k}(m + k)
    offs = nlpr.search_offsets(p.S)
    kept = [t for t, tau in enumerate(offs) if not half or tau[0] > 0 or (tau[0] == 0 and tau[1] > 0)]
    nP = len(nlpr.patch_offsets(p.K))
    sig = s[5 * img:5 * img + len(kept) * nP * img].reshape(len(kept), nP, Ls, p.H, p.W)
    assert s.size == 5 * img + len(kept) * nP * img + Ls * 2 * (2 * p.S + 1) * p.H * p.W
    for j, t in enumerate(kept):
        for kk, k in enumerate(nlpr.patch_offsets(p.K)):
            ref = nlpr.to_lhw(np.roll(st.Sig[t, kk], shift=(-k[0], -k[1]), axis=(0, 1)))
            assert np.abs(sig[j, kk] - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())


CASES = {
    # several latent row tiles with a ragged last tile, odd L_s (padded FFT pair), radix 4*2*5
    "40x40_K1S2": dict(H=40, W=40, L_l=6, L_h=2, L_s=3, K=1, S=2, iters=30),
    # 5x5 patches, 7x7 window, 9x9 blur, several tiles, radix 4*4*3 and 4*4*4
    "48x64_K2S3": dict(H=48, W=64, L_l=8, L_h=3, L_s=4, K=2, S=3, blur_size=9, blur_sigma=1.7, iters=30),
    # radix-5 and radix-3 lengths, K = 0 (pixel differences)
    "60x20_K0S1": dict(H=60, W=20, L_l=5, L_h=2, L_s=2, K=0, S=1, iters=25),
    # lambda2 = 0 (the latent pass still runs: Sigma stays 0, G = D X)
    "32x32_lam0": dict(H=32, W=32, L_l=4, L_h=2, L_s=2, K=1, S=1, lam2=0.0, iters=20),
    # the largest patch (7x7, K = 3)
    "36x40_K3S1": dict(H=36, W=40, L_l=4, L_h=2, L_s=2, K=3, S=1, iters=15),
}


@pytest.mark.parametrize("half", [1, 0])
@pytest.mark.parametrize("impl", [1, 0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_parity(name, impl, half):
    kw = dict(CASES[name])
    iters = kw.pop("iters")
    if impl == 1 and kw["W"] % 8:
        pytest.skip("the bulk-copy latent pass needs W to be a multiple of 8 (FP32)")
    p = small(**kw)
    g = gpu_solve(p, iters, opts=[(FUSE_OPT_LATENT_IMPL, impl), (FUSE_OPT_HALF_WINDOW, half)])
    Xo, _, _ = oracle_solve(p, iters)
    assert rel(g["X"], Xo) <= 1e-5
    Zo = np.einsum("chw,cl->lhw", Xo, p.E)
    assert rel(g["Z"], Zo) <= 1e-5


@pytest.mark.parametrize("half", [1, 0])
@pytest.mark.parametrize("impl", [1, 0])
def test_fp64_parity(impl, half):
    p = small(H=40, W=36, L_l=5, L_h=2, L_s=3, K=1, S=2)
    g = gpu_solve(p, 25, dtype="f64", wdtype="f64", opts=[(FUSE_OPT_LATENT_IMPL, impl), (FUSE_OPT_HALF_WINDOW, half)])
    Xo, _, _ = oracle_solve(p, 25)
    assert rel(g["X"], Xo) <= 1e-11


def test_identity_subspace_and_ratio2():
    p = synth.make_problem(H=24, W=24, L_l=3, L_h=2, L_s=3, d=2, blur_size=3, blur_sigma=0.8, K=1, S=1,
                           lam1=0.7, lam2=2e-2, rho=0.1, h=0.4, seed=5, E_identity=True)
    g = gpu_solve(p, 20)
    Xo, _, _ = oracle_solve(p, 20)
    assert rel(g["X"], Xo) <= 1e-5


def test_bf16_weights_parity_with_shared_weights():
    # The oracle's FP64 weights rounded to bf16 are loaded into both sides.
    p = small(H=64, W=64, L_l=10, L_h=4, L_s=5, K=2, S=3, blur_size=9, blur_sigma=1.7)
    om = nlpr.round_bf16(nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h))
    g = gpu_solve(p, 40, wdtype="bf16", omega=om)
    Xo, _, _ = oracle_solve(p, 40, omega=om)
    assert rel(g["X"], Xo) <= 1e-5


def test_iters_zero_returns_zero():
    p = small()
    g = gpu_solve(p, 0)
    assert not np.any(g["X"])


def test_graph_and_direct_launch_bitwise_equal():
    p = small()
    a = gpu_solve(p, 12, graph=True)["X"]
    b = gpu_solve(p, 12, graph=False)["X"]
    assert np.array_equal(a, b)


def test_run_to_run_deterministic():
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4)
    a = gpu_solve(p, 10)["X"]
    b = gpu_solve(p, 10)["X"]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("threads,stages,bands", [(32, 2, 1), (64, 3, 3), (256, 4, 2), (128, 16, 1), (256, 8, 4),
                                                   (256, 6, 64)])
def test_latent_ring_shapes_bitwise_equal(threads, stages, bands):
    # The pipelined latent pass gives bit-identical results for every block / ring shape and
    # matches the register-staged form (same arithmetic per element, same summation order).
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4, blur_size=9, blur_sigma=1.7)
    ref = gpu_solve(p, 6, opts=[(FUSE_OPT_LATENT_IMPL, 0)])["X"]          # default: half window
    got = gpu_solve(p, 6, opts=[(FUSE_OPT_LATENT_IMPL, 1), (FUSE_OPT_LATENT_THREADS, threads),
                                (FUSE_OPT_LATENT_STAGES, stages), (FUSE_OPT_LATENT_BANDS, bands)])["X"]
    assert np.array_equal(got, ref)


def test_objective_matches_oracle():
    # fuse_objective: 1/2||Y_l - SBXE||^2, lambda1/2||Y_h - XER||^2, lambda2 phi(X), ||X||^2 at the
    # final X, against the oracle's terms evaluated at the oracle's X (FP32 iterates: 1e-5).
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4, blur_size=9, blur_sigma=1.7)
    g = gpu_solve(p, 15)
    obj = g["f"].objective(g["yl"], g["yh"])
    Xo, _, om = oracle_solve(p, 15)
    X = nlpr.to_hwl(Xo)
    Yl, Yh = nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh)
    r1 = nlpr.mat(Yl) - nlpr.mat(nlpr.decimate(nlpr.blur(X, p.blur), p.d)) @ p.E
    r2 = nlpr.mat(Yh) - nlpr.mat(X) @ p.E @ p.R
    ref = [0.5 * (r1 ** 2).sum(), 0.5 * p.lam1 * (r2 ** 2).sum(), p.lam2 * nlpr.nlpr(X, om, p.K, p.S),
           (X ** 2).sum()]
    for a, b in zip(obj, ref):
        assert abs(a - b) <= 2e-5 * abs(b)
    total = sum(obj[:3])
    assert abs(total - nlpr.objective(X, Yl, Yh, p.blur, p.d, p.R, p.E, om, p.K, p.S, p.lam1, p.lam2)) <= 2e-5 * total


def test_checkpoint_resume_bitwise():
    # fuse_get_state / fuse_set_state: stopping after 5 iterations and resuming for 7 more gives
    # the same bits as 12 uninterrupted iterations.
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4)
    full = gpu_solve(p, 12)["X"]
    a = gpu_solve(p, 5)
    f = a["f"]
    st = f.get_state()
    f2 = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    f2.weights(a["yh"])
    f2.set_state(st)
    X, _ = f2.solve(a["yl"], a["yh"], 7, warm=True)
    f2.sync()
    assert np.array_equal(X.double().cpu().numpy(), full)


def test_run_host_matches_device_path():
    from paper_2210_04184_gb300.fuse import fuse_run_host
    p = small()
    g = gpu_solve(p, 10)
    f = g["f"]
    Yl = np.ascontiguousarray(p.Yl, dtype=np.float32)
    Yh = np.ascontiguousarray(p.Yh, dtype=np.float32)
    X = np.zeros((p.L_s, p.H, p.W), dtype=np.float32)
    Z = np.zeros((p.L_l, p.H, p.W), dtype=np.float32)
    fuse_run_host(f.ctx, Yl.ctypes.data, Yh.ctypes.data, None, 10, X.ctypes.data, Z.ctypes.data)
    assert np.array_equal(X.astype(np.float64), g["X"])
    assert np.array_equal(Z.astype(np.float64), g["Z"])


def test_half_window_equals_full_window():
    # The half-window state reproduces the full-window iterates up to summation order.
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4, blur_size=9, blur_sigma=1.7)
    a = gpu_solve(p, 30, opts=[(FUSE_OPT_HALF_WINDOW, 0)])["X"]
    b = gpu_solve(p, 30, opts=[(FUSE_OPT_HALF_WINDOW, 1)])["X"]
    assert rel(b, a) <= 2e-6
    a64 = gpu_solve(p, 30, dtype="f64", wdtype="f64", opts=[(FUSE_OPT_HALF_WINDOW, 0)])["X"]
    b64 = gpu_solve(p, 30, dtype="f64", wdtype="f64", opts=[(FUSE_OPT_HALF_WINDOW, 1)])["X"]
    assert rel(b64, a64) <= 1e-13


def test_contexts_of_different_sizes_coexist():
    # Kernel shared-memory caps are process-wide: a small context created after a large one
    # must not break the large one's launches.
    big = small(H=96, W=96, L_l=6, L_h=2, L_s=3)
    little = small(H=24, W=20, L_l=6, L_h=2, L_s=3, K=0, S=1, blur_size=3)
    fb = Fusion.from_problem(big, dtype="f32", wdtype="f32")
    fl = Fusion.from_problem(little, dtype="f32", wdtype="f32")
    for f, p in ((fb, big), (fl, little)):
        f.weights(torch.tensor(p.Yh, dtype=torch.float32, device="cuda"))
        X, _ = f.solve(torch.tensor(p.Yl, dtype=torch.float32, device="cuda"),
                       torch.tensor(p.Yh, dtype=torch.float32, device="cuda"), 4)
        f.sync()
        assert torch.isfinite(X).all()


def test_autotune_and_fft_shapes_keep_results():
    # Launch shapes never change the arithmetic: results are bit-identical after the tuner and
    # for every FFT tile shape.
    from paper_2210_04184_gb300.fuse import FUSE_OPT_FFT_ROWS, FUSE_OPT_FFT_COLS
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4, blur_size=9, blur_sigma=1.7)
    ref = gpu_solve(p, 8)["X"]
    for r, cw in ((1, 2), (2, 16), (8, 4)):
        got = gpu_solve(p, 8, opts=[(FUSE_OPT_FFT_ROWS, r), (FUSE_OPT_FFT_COLS, cw)])["X"]
        assert np.array_equal(got, ref)
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
    f.weights(yh)
    chosen = f.autotune(yl, yh, iters=1)
    assert chosen["latent_threads"] in (128, 192, 256) and chosen["fft_rows"] in (1, 2, 4, 8)
    X, _ = f.solve(yl, yh, 8)
    f.sync()
    assert np.array_equal(X.double().cpu().numpy(), ref)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_more_than_32_subspace_bands(dtype):
    # E = I with 40 bands: the pixel updates take the shared-memory path for L_s > 32
    p = synth.make_problem(H=24, W=32, L_l=40, L_h=3, L_s=40, d=4, blur_size=5, blur_sigma=1.0, K=1, S=2,
                           lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=9, E_identity=True)
    assert p.L_s == 40
    g = gpu_solve(p, 15, dtype=dtype, wdtype=dtype)
    Xo, _, _ = oracle_solve(p, 15)
    assert rel(g["X"], Xo) <= (1e-5 if dtype == "f32" else 1e-11)
    assert rel(g["Z"], np.einsum("chw,cl->lhw", Xo, p.E)) <= (1e-5 if dtype == "f32" else 1e-11)


def test_identity_subspace_at_93_bands():
    # the HS+MS bands with E = I (L_s = 93, the secondary form of that workload) on a 64 x 64 crop
    p = synth.make_problem(H=64, W=64, L_l=93, L_h=4, L_s=93, d=4, blur_size=9, blur_sigma=1.7, K=2, S=3,
                           snr_l=35.0, snr_h=35.0, kind="hsms", seed=10, E_identity=True)
    om = nlpr.round_bf16(nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h))
    g = gpu_solve(p, 4, dtype="f32", wdtype="bf16", omega=om)
    Xo, _, _ = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S, p.lam1, p.lam2,
                         p.rho, om, 4, fast=True, inplace=True)
    assert rel(g["X"], nlpr.to_lhw(Xo)) <= 1e-5


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_non_separable_square_blur(dtype):
    # random 5x5 taps (rank 5): the 2D square-blur stencil, against the oracle's direct convolution
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4)
    rng = np.random.default_rng(77)
    p.blur = rng.random((5, 5))
    p.blur /= p.blur.sum()
    wd = "f64" if dtype == "f64" else "f32"
    g = gpu_solve(p, 10, dtype=dtype, wdtype=wd)
    Xo, _, _ = oracle_solve(p, 10)
    assert rel(g["X"], Xo) <= (1e-11 if dtype == "f64" else 1e-5)


@pytest.mark.parametrize("bsize,sigma,Ls", [(9, 1.7, 4), (5, 1.0, 4), (11, 2.0, 4), (3, 0.8, 4), (9, 1.7, 5)])
def test_separable_blur_equals_2d_stencil(bsize, sigma, Ls):
    # a Gaussian blur factors as cu(u) cv(v): the separable passes and the 2D stencil apply the same
    # operator up to rounding (FP64, 12 iterations); the separable path also matches the oracle.
    # L_s = 5 leaves the last block of the several-bands-per-block B X kernel one band.
    from paper_2210_04184_gb300.fuse import FUSE_OPT_SEPARABLE_BLUR
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=Ls, blur_size=bsize, blur_sigma=sigma)
    a = gpu_solve(p, 12, dtype="f64", wdtype="f64")["X"]
    b = gpu_solve(p, 12, dtype="f64", wdtype="f64", opts=[(FUSE_OPT_SEPARABLE_BLUR, 0)])["X"]
    assert rel(a, b) <= 1e-13
    Xo, _, _ = oracle_solve(p, 12)
    assert rel(a, Xo) <= 1e-11
