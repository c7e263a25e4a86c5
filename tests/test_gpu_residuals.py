"""ADMM residual norms of the last iteration of a solve (FUSE_OPT_RESIDUALS, fuse_residuals)
against the oracle's (nlpr.residuals, computed from the stored consecutive iterates): primal
sqrt(||BX - P1||^2 + ||X - P2||^2 + sum ||D X - Q||^2) and dual
rho ||B^T dP1 + dP2 + sum D^T dQ|| (Sec. IV, scaled form of the splitting of eq. fusionoptim).
FP64 within 1e-9 relative; FP32 within 1e-5 of the scale of the terms (the norms are differences
of consecutive iterates, so FP32 rounding of the iterates enters at the iterates' scale)."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300 import fuse  # noqa: E402
from paper_2210_04184_gb300.fuse import (Fusion, FuseError, FUSE_OPT_RESIDUALS, FUSE_OPT_HALF_WINDOW,  # noqa: E402
                                         FUSE_OPT_GRAPH, FUSE_OPT_STATE_FORMAT)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def small(**kw):
    base = dict(H=48, W=64, L_l=8, L_h=3, L_s=4, d=4, blur_size=9, blur_sigma=1.7, K=2, S=3,
                lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=31)
    base.update(kw)
    return synth.make_problem(**base)


def oracle_residuals(p, iters, om, warm_split=None):
    """(primal, dual) of iteration `iters` and the scales of the quantities they difference."""
    Yl, Yh = nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh)
    keep = {}

    def cb(st, su):
        if st.t in (iters - 1, iters):
            keep[st.t] = st.copy()

    _, st, su = nlpr.admm(Yl, Yh, p.blur, p.d, p.R, p.E, p.K, p.S, p.lam1, p.lam2, p.rho, om, iters,
                          fast=True, callback=cb)
    prev = keep.get(iters - 1) or nlpr.State.zeros(p.H, p.W, p.L_s, p.K, p.S)
    r = nlpr.residuals(prev, keep[iters], su)
    s = keep[iters]
    dual_terms = nlpr.blur_t(s.P1, p.blur) + s.P2 + nlpr.dt_sum(s.Q, np.zeros_like(s.Q), p.K, p.S)
    scale_p = float(np.sqrt((s.Lam1 ** 2).sum() + (s.Lam2 ** 2).sum() + (s.Sig ** 2).sum()))
    scale_d = p.rho * float(np.sqrt((dual_terms ** 2).sum()))
    return r, (scale_p, scale_d)


def gpu_residuals(p, iters, dtype, wdtype="f32", opts=(), om=None, splits=None):
    td = torch.float64 if dtype == "f64" else torch.float32
    f = Fusion.from_problem(p, dtype=dtype, wdtype=wdtype)
    for o, v in opts:
        f.set_option(o, v)
    f.set_option(FUSE_OPT_RESIDUALS, 1)
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    if om is not None:
        f.set_weights(torch.tensor(om, dtype=f.wtdtype, device="cuda"))
    else:
        f.weights(yh)
    if splits:
        warm = False
        for k in splits:
            X, _ = f.solve(yl, yh, k, warm=warm)
            warm = True
    else:
        X, _ = f.solve(yl, yh, iters)
    r = f.residuals()
    return r, X, f, yl, yh


@pytest.mark.parametrize("iters", [1, 2, 3, 12])
@pytest.mark.parametrize("half", [1, 0])
def test_residuals_fp64(iters, half):
    p = small()
    om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    (rp, rd), _ = oracle_residuals(p, iters, om)
    (gp, gd), _, f, _, _ = gpu_residuals(p, iters, "f64", "f64", opts=[(FUSE_OPT_HALF_WINDOW, half)], om=om)
    assert abs(gp - rp) <= 1e-9 * rp
    assert abs(gd - rd) <= 1e-9 * max(rd, 1e-300)
    f.close()


@pytest.mark.parametrize("case", ["base", "ratio2_identity", "odd_bands_k0"])
def test_residuals_fp32(case):
    kw = {"base": {}, "ratio2_identity": dict(d=2, L_l=4, L_s=4, E_identity=True, K=1, S=2, H=40, W=40),
          "odd_bands_k0": dict(L_s=5, K=0, S=2, W=40)}[case]
    p = small(**kw)
    om = nlpr.round_bf16(nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h))
    for iters in (2, 9):
        (rp, rd), (sp, sd) = oracle_residuals(p, iters, om)
        (gp, gd), _, f, _, _ = gpu_residuals(p, iters, "f32", "bf16", om=om)
        assert abs(gp - rp) <= 1e-5 * (rp + sp), (gp, rp, sp)
        assert abs(gd - rd) <= 1e-5 * (rd + sd), (gd, rd, sd)
        f.close()


def test_residuals_of_a_warm_continuation():
    # solves of 4 + 3 + 5 iterations continuing from each other report iteration 12's residuals
    p = small()
    om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    (rp, rd), _ = oracle_residuals(p, 12, om)
    (gp, gd), _, f, _, _ = gpu_residuals(p, 12, "f64", "f64", om=om, splits=[4, 3, 5])
    assert abs(gp - rp) <= 1e-9 * rp and abs(gd - rd) <= 1e-9 * rd
    f.close()


def test_monitor_leaves_iterates_unchanged():
    # the monitored last iteration gives the same bits as a plain one, graphs on or off
    p = small()
    f0 = Fusion.from_problem(p, dtype="f32", wdtype="bf16")
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
    f0.weights(yh)
    X0, _ = f0.solve(yl, yh, 10)
    for graph in (1, 0):
        _, X1, f1, _, _ = gpu_residuals(p, 10, "f32", "bf16", opts=[(FUSE_OPT_GRAPH, graph)])
        assert torch.equal(X0, X1)
        f1.close()
    f0.close()


def test_residuals_decrease_towards_the_limit():
    # both norms fall by orders of magnitude over a long run (the iterates converge, Theorem 1)
    p = small(H=32, W=32, K=1, S=1)
    r10, _, f, yl, yh = gpu_residuals(p, 10, "f64", "f64")
    f.solve(yl, yh, 3000, warm=True)
    r3k = f.residuals()
    assert r3k[0] < 1e-2 * r10[0] and r3k[1] < 1e-2 * r10[1]
    f.close()


def test_residual_errors():
    p = small()
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
    f.weights(yh)
    f.solve(yl, yh, 3)
    with pytest.raises(FuseError) as e:               # monitor off
        f.residuals()
    assert e.value.status == fuse.FUSE_ESTATE
    fuse.fuse_reset_error(f.ctx)
    f.set_option(FUSE_OPT_RESIDUALS, 1)
    f.solve(yl, yh, 3)
    f.residuals()
    f.weights(yh)                                     # inputs changed since the monitored iteration
    with pytest.raises(FuseError) as e:
        f.residuals()
    assert e.value.status == fuse.FUSE_ESTATE
    fuse.fuse_reset_error(f.ctx)
    # a NaN in Y_l reaches the scaled duals: FUSE_ENONFINITE
    bad = yl.clone()
    bad[0, 0, 0] = float("nan")
    f.solve(bad, yh, 4)
    with pytest.raises(FuseError) as e:
        f.residuals()
    assert e.value.status == fuse.FUSE_ENONFINITE
    fuse.fuse_reset_error(f.ctx)
    f.close()
    # the 16-bit state is not monitored
    g = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    g.set_option(FUSE_OPT_STATE_FORMAT, 1)
    with pytest.raises(FuseError) as e:
        g.set_option(FUSE_OPT_RESIDUALS, 1)
    assert e.value.status == fuse.FUSE_EUNSUPPORTED
    g.close()
