"""The X update with S B kept in the X system (FUSE_OPT_X_UPDATE = 1) against the oracle's
variant (nlpr.admm(..., x_update="sb")), which solves every alias class as a dense d^2 x d^2
system; the CUDA path solves it in closed form (Sherman-Morrison) inside the column FFT pass.

Cases span ratios 1 to 4 (classes of 1 to 16 frequencies), mixed-radix sizes, square and
non-square asymmetric blurs (a complex b^, so a dropped conjugate shows), E E^T = eps I with
eps != 1, half and full window, K = 0..2 and the 16-bit state.  Tolerances as in the parity
tests: FP32 1e-5 relative, FP64 1e-11."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300.fuse import (Fusion, FusionBatch, FuseError, FUSE_EUNSUPPORTED,  # noqa: E402
                                         FUSE_OPT_HALF_WINDOW, FUSE_OPT_STATE_FORMAT, FUSE_OPT_X_UPDATE,
                                         fuse_get_option, fuse_reset_error)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def problem(H=40, W=48, d=4, L_s=3, K=1, S=2, blur=(5, 5), seed=81, E_scale=1.0, L_l=6, **kw):
    p = synth.make_problem(H=H, W=W, L_l=L_l, L_h=2, L_s=L_s, d=d, blur_size=5, blur_sigma=1.0, K=K, S=S,
                           lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=seed, **kw)
    rng = np.random.default_rng(seed + 1)
    k = rng.random(blur) + 0.2                      # asymmetric: b^ is complex
    p.blur = k / k.sum()
    p.E = p.E * E_scale
    return p


def gpu(p, iters, omega, dtype="f32", opts=()):
    td = torch.float64 if dtype == "f64" else torch.float32
    f = Fusion.from_problem(p, dtype=dtype, wdtype=dtype)
    for o, v in ((FUSE_OPT_X_UPDATE, 1),) + tuple(opts):
        f.set_option(o, v)
    f.set_weights(torch.tensor(omega, dtype=td, device="cuda"))
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    X, Z = f.solve(yl, yh, iters, want_Z=True)
    f.sync()
    return X.double().cpu().numpy(), Z.double().cpu().numpy(), f


def oracle(p, iters, omega, levels=None):
    X, st, _ = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S, p.lam1, p.lam2,
                         p.rho, omega, iters, fast=True, x_update="sb", state_levels=levels)
    return nlpr.to_lhw(X)


def omega_of(p, dtype):
    om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    return om.astype(np.float32).astype(np.float64) if dtype == "f32" else om


@pytest.mark.parametrize("case", [
    dict(),                                                     # d 4: 16 frequencies per class
    dict(H=48, W=40, d=2, K=2, S=3, blur=(3, 3), seed=82),
    dict(H=36, W=48, d=3, blur=(3, 5), seed=83),                # radix 3, non-square blur
    dict(H=30, W=40, d=1, K=0, blur=(5, 3), seed=84),           # classes of one frequency
    dict(E_scale=1.7, seed=85),                                  # E E^T = 2.89 I
    dict(H=64, W=96, d=4, L_s=5, K=1, S=1, seed=86),            # several blocks per band pair, odd L_s
    # 49 band pairs: two base columns per block and W/d = 25, so the last block is half masked
    dict(H=40, W=100, d=4, L_l=100, L_s=98, K=0, S=1, blur=(3, 3), seed=91),
])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_sb_update_matches_oracle(case, dtype):
    p = problem(**case)
    om = omega_of(p, dtype)
    X, Z, _ = gpu(p, 20, om, dtype)
    Xo = oracle(p, 20, om)
    tol = 1e-5 if dtype == "f32" else 1e-11
    assert rel(X, Xo) <= tol
    assert rel(Z, np.einsum("chw,cl->lhw", Xo, p.E)) <= tol


def test_sb_update_full_window_and_fixed_point_state():
    p = problem(seed=87)
    om = omega_of(p, "f32")
    Xo = oracle(p, 15, om)
    X, _, _ = gpu(p, 15, om, opts=((FUSE_OPT_HALF_WINDOW, 0),))
    assert rel(X, Xo) <= 1e-5
    X16, _, _ = gpu(p, 15, om, opts=((FUSE_OPT_STATE_FORMAT, 1),))
    assert rel(X16, oracle(p, 15, om, levels=32767)) <= 1e-5


def test_sb_update_differs_from_the_paper_splitting_and_switches_back():
    p = problem(seed=88)
    om = omega_of(p, "f32")
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    f.set_weights(torch.tensor(om, dtype=torch.float32, device="cuda"))
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
    X0, _ = f.solve(yl, yh, 10)
    X0 = X0.clone()
    f.set_option(FUSE_OPT_X_UPDATE, 1)
    assert fuse_get_option(f.ctx, FUSE_OPT_X_UPDATE) == 1
    X1, _ = f.solve(yl, yh, 10)
    X1 = X1.clone()
    f.set_option(FUSE_OPT_X_UPDATE, 0)
    X2, _ = f.solve(yl, yh, 10)
    f.sync()
    assert torch.equal(X2, X0)                       # the paper's iterates again, bit for bit
    assert rel(X1.double().cpu().numpy(), X0.double().cpu().numpy()) > 1e-4   # other iterates


def test_sb_update_refusals():
    p = problem(d=1, H=32, W=32, seed=89)
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    f.set_mask(np.ones((p.H, p.W), dtype=np.uint8))
    with pytest.raises(FuseError) as e:
        f.set_option(FUSE_OPT_X_UPDATE, 1)
    assert e.value.status == FUSE_EUNSUPPORTED
    fuse_reset_error(f.ctx)
    f.set_mask(None)
    f.set_option(FUSE_OPT_X_UPDATE, 1)
    with pytest.raises(FuseError) as e:
        f.set_mask(np.ones((p.H, p.W), dtype=np.uint8))
    assert e.value.status == FUSE_EUNSUPPORTED
    fuse_reset_error(f.ctx)
    # the reverse pass and batches follow the paper's splitting
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
    f.weights(yh)
    with pytest.raises(FuseError) as e:
        f.grad_forward(yl, yh, 2)
    assert e.value.status == FUSE_EUNSUPPORTED
    fuse_reset_error(f.ctx)
    with pytest.raises(FuseError) as e:
        FusionBatch([f])
    assert e.value.status == FUSE_EUNSUPPORTED
    # E with unequal row norms: E E^T is not a multiple of I
    q = problem(seed=90)
    q.E = q.E * np.array([1.0, 2.0, 1.0])[:, None]
    g = Fusion.from_problem(q, dtype="f32", wdtype="f32")
    with pytest.raises(FuseError) as e:
        g.set_option(FUSE_OPT_X_UPDATE, 1)
    assert e.value.status == FUSE_EUNSUPPORTED
