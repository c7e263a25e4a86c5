"""Batched solves of problems with uneven sizes (one launch per ADMM phase over all problems):
bit-identical to solving each problem alone, and within the FP32 tolerance of the oracle."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300 import fuse  # noqa: E402
from paper_2210_04184_gb300.fuse import Fusion, FusionBatch, FuseError  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def _problems(dtype):
    sizes = [(40, 40), (48, 64), (96, 96), (32, 24), (60, 120)]
    return [synth.make_problem(H=h, W=w, L_l=9, L_h=3, L_s=5, d=4, blur_size=5, blur_sigma=1.0, K=1, S=2,
                               lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=100 + i)
            for i, (h, w) in enumerate(sizes)]


def _contexts(ps, dtype, wdtype):
    td = torch.float64 if dtype == "f64" else torch.float32
    fs, yl, yh = [], [], []
    for p in ps:
        f = Fusion.from_problem(p, dtype=dtype, wdtype=wdtype)
        yl.append(torch.tensor(p.Yl, dtype=td, device="cuda"))
        yh.append(torch.tensor(p.Yh, dtype=td, device="cuda"))
        f.weights(yh[-1])
        fs.append(f)
    return fs, yl, yh


@pytest.mark.parametrize("dtype,wdtype", [("f32", "bf16"), ("f32", "f32"), ("f64", "f64")])
def test_batch_equals_single_solves(dtype, wdtype):
    ps = _problems(dtype)
    fs, yl, yh = _contexts(ps, dtype, wdtype)
    single = []
    for f, a, b in zip(fs, yl, yh):
        X, Z = f.solve(a, b, 12, want_Z=True)
        f.sync()
        single.append((X.clone(), Z.clone()))
    batch = FusionBatch(fs)
    Xs, Zs = batch.solve(yl, yh, 12, want_Z=True)
    batch.sync()
    for (X, Z), Xb, Zb in zip(single, Xs, Zs):
        assert torch.equal(X, Xb) and torch.equal(Z, Zb)
    batch.close()


def test_batch_matches_oracle_and_graph_replay():
    ps = _problems("f32")
    fs, yl, yh = _contexts(ps, "f32", "f32")
    batch = FusionBatch(fs)
    Xs, _ = batch.solve(yl, yh, 20)
    batch.sync()
    batch.set_option(fuse.FUSE_OPT_GRAPH, 0)
    Xd, _ = batch.solve(yl, yh, 20)
    batch.sync()
    for a, b in zip(Xs, Xd):
        assert torch.equal(a, b)
    for i in (1, 4):
        p = ps[i]
        om = nlpr.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
        Xo, _, _ = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S,
                             p.lam1, p.lam2, p.rho, om, 20, fast=True)
        Xo = nlpr.to_lhw(Xo)
        err = np.linalg.norm(Xs[i].double().cpu().numpy() - Xo) / np.linalg.norm(Xo)
        assert err <= 1e-5


@pytest.mark.parametrize("threads,stages,bands", [(64, 3, 1), (256, 8, 2), (128, 4, 5)])
def test_batch_ring_shapes(threads, stages, bands):
    ps = _problems("f32")
    fs, yl, yh = _contexts(ps, "f32", "f32")
    batch = FusionBatch(fs)
    ref, _ = batch.solve(yl, yh, 6)
    batch.sync()
    ref = [r.clone() for r in ref]
    batch.set_option(fuse.FUSE_OPT_LATENT_THREADS, threads)
    batch.set_option(fuse.FUSE_OPT_LATENT_STAGES, stages)
    batch.set_option(fuse.FUSE_OPT_LATENT_BANDS, bands)
    got, _ = batch.solve(yl, yh, 6)
    batch.sync()
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_batch_rejects_mismatched_contexts():
    a = synth.make_problem(H=40, W=40, L_l=9, L_h=3, L_s=5, d=4, blur_size=5, K=1, S=2, seed=1)
    b = synth.make_problem(H=40, W=40, L_l=9, L_h=3, L_s=5, d=4, blur_size=5, K=2, S=2, seed=2)
    fa = Fusion.from_problem(a, dtype="f32", wdtype="f32")
    fb = Fusion.from_problem(b, dtype="f32", wdtype="f32")
    with pytest.raises(FuseError) as e:
        FusionBatch([fa, fb])
    assert e.value.status == fuse.FUSE_EINVAL
    with pytest.raises(FuseError):
        FusionBatch([fa, fa])


def test_batch_autotune_keeps_results():
    ps = _problems("f32")
    fs, yl, yh = _contexts(ps, "f32", "bf16")
    batch = FusionBatch(fs)
    ref, _ = batch.solve(yl, yh, 5)
    batch.sync()
    ref = [r.clone() for r in ref]
    batch.autotune(yl, yh, iters=1)
    got, _ = batch.solve(yl, yh, 5)
    batch.sync()
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


def test_batch64_full_size_sampled():
    # the batched workload at its full size (64 problems of 96..384 pixels a side, 100
    # iterations, BF16 weights) in the bench's launch configuration: every problem finite,
    # sampled problems equal to their single-problem solves bit for bit, and the smallest
    # against the oracle (with the GPU's BF16 weights)
    ps = synth.batch_workload(64)
    iters = ps[0].iters
    fs, yl, yh = _contexts(ps, "f32", "bf16")
    batch = FusionBatch(fs)
    batch.autotune(yl, yh, iters=1)
    Xs, _ = batch.solve(yl, yh, iters)
    batch.sync()
    for X in Xs:
        assert bool(torch.isfinite(X).all())
    order = sorted(range(len(ps)), key=lambda i: ps[i].H)
    for i in (order[0], order[len(order) // 2], order[-1]):
        X, _ = fs[i].solve(yl[i], yh[i], iters)
        fs[i].sync()
        assert torch.equal(X, Xs[i])
    i = order[0]
    p = ps[i]
    om = fs[i].get_weights().double().cpu().numpy()
    Xo, _, _ = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S, p.lam1, p.lam2,
                         p.rho, om, iters, fast=True, inplace=True)
    Xg = Xs[i].double().cpu().numpy()
    assert np.linalg.norm(Xg - nlpr.to_lhw(Xo)) / np.linalg.norm(Xo) <= 1e-5
    batch.close()


def test_batch_with_different_blur_taps():
    # problems with the same blur size but different taps (sigma 1.0 and 1.6): the batch falls back
    # to the 2D stencil that reads each problem's taps, and every problem equals its single solve
    # with the 2D stencil (a single Gaussian blur otherwise takes the separable passes: the same
    # operator with another rounding)
    ps = [synth.make_problem(H=h, W=w, L_l=9, L_h=3, L_s=5, d=4, blur_size=5, blur_sigma=sg, K=1, S=2,
                             lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=300 + i)
          for i, (h, w, sg) in enumerate([(40, 40, 1.0), (48, 64, 1.6), (32, 24, 1.0)])]
    fs, yl, yh = _contexts(ps, "f32", "f32")
    single = []
    for f, a, b in zip(fs, yl, yh):
        f.set_option(fuse.FUSE_OPT_SEPARABLE_BLUR, 0)
        X, _ = f.solve(a, b, 9)
        f.sync()
        single.append(X.clone())
        f.set_option(fuse.FUSE_OPT_SEPARABLE_BLUR, 1)
    batch = FusionBatch(fs)
    Xs, _ = batch.solve(yl, yh, 9)
    batch.sync()
    for X, Xb in zip(single, Xs):
        assert torch.equal(X, Xb)
    batch.close()
