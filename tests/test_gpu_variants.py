"""Variants of the method on the same kernels, against the oracle run the same way.

- ablation regularisers: omega = 1 (no guide), pixel differences K = 0 with and without guide
  weights, and local 4-neighbour differences with omega = 1 (anisotropic TV: the diagonal
  offsets of the 3x3 window get weight 0, which leaves them unpenalised);
- a general sampling operator S given as a pixel mask (guided inpainting): parity of the
  iterates, the objective and the reverse pass; the d = 2 lattice given as a mask reproduces the
  regular d = 2 solve bit for bit.
Tolerances as in the parity tests: FP32 1e-5 relative, FP64 1e-11 (reverse pass 1e-9)."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import grad as ograd, nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300.fuse import (Fusion, FusionBatch, FuseError, FUSE_EINVAL,  # noqa: E402
                                         FUSE_OPT_HALF_WINDOW, fuse_reset_error)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def small(**kw):
    base = dict(H=40, W=40, L_l=6, L_h=2, L_s=3, d=4, blur_size=5, blur_sigma=1.0, K=1, S=2,
                lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=41)
    base.update(kw)
    return synth.make_problem(**base)


def run(p, iters, omega, dtype="f32", mask=None, opts=()):
    td = torch.float64 if dtype == "f64" else torch.float32
    f = Fusion.from_problem(p, dtype=dtype, wdtype=dtype)
    for o, v in opts:
        f.set_option(o, v)
    if mask is not None:
        f.set_mask(mask)
    f.set_weights(torch.tensor(omega, dtype=td, device="cuda"))
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    X, Z = f.solve(yl, yh, iters, want_Z=True)
    f.sync()
    return X.double().cpu().numpy(), Z.double().cpu().numpy(), f, yl, yh


def oracle(p, iters, omega, mask=None):
    X, _, _ = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S, p.lam1, p.lam2,
                        p.rho, omega, iters, fast=True, mask=None if mask is None else mask.astype(float))
    return nlpr.to_lhw(X)


def four_neighbour_weights(S, H, W):
    om = np.zeros((len(nlpr.search_offsets(S)), H, W))
    for t, tau in enumerate(nlpr.search_offsets(S)):
        if abs(tau[0]) + abs(tau[1]) == 1:
            om[t] = 1.0
    return om


@pytest.mark.parametrize("variant", ["omega1", "pixel_guided", "pixel_omega1", "local_tv"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_ablation_variants_match_oracle(variant, dtype):
    K = 1 if variant == "omega1" else 0
    S = 1 if variant == "local_tv" else 2
    p = small(K=K, S=S, lam2=5e-2)
    nW = len(nlpr.search_offsets(S))
    if variant in ("omega1", "pixel_omega1"):
        om = np.ones((nW, p.H, p.W))
    elif variant == "pixel_guided":
        om = nlpr.weights(nlpr.to_hwl(p.Yh), 0, S, p.h)
    else:
        om = four_neighbour_weights(S, p.H, p.W)
    if dtype == "f32":
        om = om.astype(np.float32).astype(np.float64)
    X, Z, _, _, _ = run(p, 30, om, dtype)
    Xo = oracle(p, 30, om)
    tol = 1e-5 if dtype == "f32" else 1e-11
    assert rel(X, Xo) <= tol
    assert rel(Z, np.einsum("chw,cl->lhw", Xo, p.E)) <= tol


def inpainting(seed=43, blur=1, **kw):
    base = dict(H=48, W=40, L_l=6, L_h=2, L_s=4, d=1, blur_size=blur, blur_sigma=1.0, K=1, S=2,
                lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=seed)
    base.update(kw)
    p = synth.make_problem(**base)
    return p, synth.sampling_mask(p.H, p.W, 0.3, seed + 1)


@pytest.mark.parametrize("blur", [1, 5])
@pytest.mark.parametrize("half", [1, 0])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_random_mask_matches_oracle(blur, half, dtype):
    p, mask = inpainting(blur=blur)
    om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    if dtype == "f32":
        om = om.astype(np.float32).astype(np.float64)
    X, Z, f, yl, yh = run(p, 25, om, dtype, mask=mask, opts=((FUSE_OPT_HALF_WINDOW, half),))
    Xo = oracle(p, 25, om, mask)
    tol = 1e-5 if dtype == "f32" else 1e-11
    assert rel(X, Xo) <= tol
    assert rel(Z, np.einsum("chw,cl->lhw", Xo, p.E)) <= tol
    if dtype == "f64":
        obj = f.objective(yl, yh)
        ref_data = nlpr.objective(nlpr.to_hwl(Xo), nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, 1, p.R, p.E,
                                  om, p.K, p.S, p.lam1, 0.0, mask=mask.astype(float))
        assert abs(obj[0] + obj[1] - ref_data) <= 1e-9 * ref_data


def test_lattice_as_mask_equals_regular_decimation():
    # the d = 2 lattice given as a mask with Y_l placed on it (junk elsewhere) is the same solve
    p = small(d=2, H=40, W=48, seed=44)
    om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h).astype(np.float32).astype(np.float64)
    X2, Z2, _, _, _ = run(p, 12, om)
    mask = np.zeros((p.H, p.W), dtype=np.uint8)
    mask[::2, ::2] = 1
    q = synth.make_problem(H=40, W=48, L_l=6, L_h=2, L_s=3, d=2, blur_size=5, blur_sigma=1.0, K=1, S=2,
                           lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=44)
    full = np.full((q.L_l, q.H, q.W), 7.0)
    full[:, ::2, ::2] = q.Yl
    q.Yl, q.d = full, 1
    X1, Z1, _, _, _ = run(q, 12, om, mask=mask)
    assert np.array_equal(X1, X2) and np.array_equal(Z1, Z2)


def test_mask_reverse_pass_matches_oracle():
    p, mask = inpainting(seed=45, blur=3)
    om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    Wt = np.random.default_rng(46).standard_normal((p.L_s, p.H, p.W))
    f = Fusion.from_problem(p, dtype="f64", wdtype="f64")
    f.set_mask(mask)
    f.set_weights(torch.tensor(om, device="cuda"))
    yl = torch.tensor(p.Yl, device="cuda")
    yh = torch.tensor(p.Yh, device="cuda")
    f.grad_forward(yl, yh, 6)
    gl, gh, pr = f.grad_backward(Xbar=torch.tensor(Wt, device="cuda"))
    _, go = ograd.unrolled_grad(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, 1, p.R, p.E, p.K, p.S, p.lam1,
                                p.lam2, p.rho, om, 6, lambda X: nlpr.to_hwl(Wt), mask=mask.astype(float))
    gl = gl.cpu().numpy()
    assert rel(gl, nlpr.to_lhw(go["Yl"])) <= 1e-9
    assert not gl[:, mask == 0].any()
    assert rel(gh.cpu().numpy(), nlpr.to_lhw(go["Yh"])) <= 1e-9
    for k in ("lam1", "lam2", "rho"):
        assert abs(pr[k] - go[k]) <= 1e-9 * abs(go[k])


def test_mask_batch_equals_single():
    ps = [inpainting(seed=50 + i, H=h, W=w) for i, (h, w) in enumerate([(40, 40), (48, 64), (32, 24)])]
    fs, yl, yh, single = [], [], [], []
    for p, mask in ps:
        f = Fusion.from_problem(p, dtype="f32", wdtype="bf16")
        f.set_mask(mask)
        a = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
        b = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
        f.weights(b)
        X, _ = f.solve(a, b, 10)
        f.sync()
        single.append(X.clone())
        fs.append(f); yl.append(a); yh.append(b)
    batch = FusionBatch(fs)
    Xs, _ = batch.solve(yl, yh, 10)
    batch.sync()
    for X, Xb in zip(single, Xs):
        assert torch.equal(X, Xb)
    batch.close()


def test_mask_needs_ratio_one_and_can_be_cleared():
    p = small()                                      # ratio 4
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    with pytest.raises(FuseError) as e:
        f.set_mask(np.ones((p.H, p.W), dtype=np.uint8))
    assert e.value.status == FUSE_EINVAL
    fuse_reset_error(f.ctx)
    q, mask = inpainting(seed=47)
    om = nlpr.weights(nlpr.to_hwl(q.Yh), q.K, q.S, q.h).astype(np.float32).astype(np.float64)
    X0, _, g, yl, yh = run(q, 8, om)                 # d = 1, every pixel observed
    g.set_mask(mask)
    Xm, _ = g.solve(yl, yh, 8)
    g.set_mask(None)
    X1, _ = g.solve(yl, yh, 8)
    g.sync()
    assert np.array_equal(X1.double().cpu().numpy(), X0)
    assert not np.array_equal(Xm.double().cpu().numpy(), X0)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_denoising_variant(dtype):
    # S = B = I (ratio 1, 1x1 blur): guided denoising of every band with the same kernels
    p = synth.make_problem(H=40, W=48, L_l=6, L_h=2, L_s=3, d=1, blur_size=1, blur_sigma=1.0, K=1, S=2,
                           lam1=1.0, lam2=2e-2, rho=5e-2, h=0.3, seed=61)
    om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    if dtype == "f32":
        om = om.astype(np.float32).astype(np.float64)
    X, Z, _, _, _ = run(p, 25, om, dtype)
    Xo = oracle(p, 25, om)
    tol = 1e-5 if dtype == "f32" else 1e-11
    assert rel(X, Xo) <= tol and rel(Z, np.einsum("chw,cl->lhw", Xo, p.E)) <= tol
