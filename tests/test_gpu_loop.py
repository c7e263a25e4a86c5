"""The whole iteration loop replayed from captured CUDA graphs (up to 256 iterations per graph),
and cold starts whose first latent pass takes the state as zero instead of reading a cleared
buffer: both give the same bits as direct launches from a cleared state."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300.fuse import (Fusion, FusionBatch, FUSE_OPT_GRAPH, FUSE_OPT_LATENT_IMPL,  # noqa: E402
                                         FUSE_OPT_STATE_FORMAT)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def small(**kw):
    base = dict(H=40, W=40, L_l=6, L_h=2, L_s=3, d=4, blur_size=5, blur_sigma=1.0, K=1, S=2,
                lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=3)
    base.update(kw)
    return synth.make_problem(**base)


def ctx(p, graph=True, opts=()):
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    if not graph:
        f.set_option(FUSE_OPT_GRAPH, 0)
    for o, v in opts:
        f.set_option(o, v)
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
    f.weights(yh)
    return f, yl, yh


def run(f, yl, yh, iters, warm=False):
    X, _ = f.solve(yl, yh, iters, warm=warm)
    f.sync()
    return X.cpu().numpy()


def test_long_solve_replays_chunked_graphs_bitwise():
    # 300 iterations: one captured loop of 256 iterations and one of 44
    p = small()
    fg, yl, yh = ctx(p)
    fd, _, _ = ctx(p, graph=False)
    assert np.array_equal(run(fg, yl, yh, 300), run(fd, yl, yh, 300))


def test_loop_cache_with_mixed_lengths():
    # solves of several lengths on one context (two cached loops, least recently used replaced),
    # cold and warm, each equal to the same sequence with direct launches
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4)
    fg, yl, yh = ctx(p)
    fd, _, _ = ctx(p, graph=False)
    for iters, warm in [(5, False), (12, False), (5, True), (7, False), (12, True), (3, True), (12, False)]:
        assert np.array_equal(run(fg, yl, yh, iters, warm), run(fd, yl, yh, iters, warm)), (iters, warm)


@pytest.mark.parametrize("opts", [(), ((FUSE_OPT_LATENT_IMPL, 0),), ((FUSE_OPT_STATE_FORMAT, 1),)])
def test_cold_start_ignores_stale_state(opts):
    # a latent state full of other values (set through fuse_set_state) does not reach a cold solve
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4)
    ref_f, yl, yh = ctx(p, opts=opts)
    ref = run(ref_f, yl, yh, 9)
    f, _, _ = ctx(p, opts=opts)
    run(f, yl, yh, 4)
    st = f.get_state()
    img = p.H * p.W * p.L_s * 4
    g = torch.Generator(device="cuda").manual_seed(1)
    st[5 * img:] = torch.randint(0, 255, (st.numel() - 5 * img,), dtype=torch.uint8, device="cuda", generator=g)
    f.set_state(st)
    assert np.array_equal(run(f, yl, yh, 9), ref)
    # graphs off: the same
    f.set_option(FUSE_OPT_GRAPH, 0)
    f.set_state(st)
    assert np.array_equal(run(f, yl, yh, 9), ref)


def test_cold_start_equals_cleared_state():
    # cold solve (first latent pass reads nothing) == zero iterations (which clears the state)
    # followed by a warm solve that reads the cleared state
    p = small(K=2, S=3, H=48, W=64, L_l=8, L_h=3, L_s=4)
    f, yl, yh = ctx(p)
    cold = run(f, yl, yh, 10)
    run(f, yl, yh, 0)
    assert np.array_equal(run(f, yl, yh, 10, warm=True), cold)


def _batch(n=4):
    sizes = [(40, 40), (48, 64), (32, 24), (64, 32)][:n]
    ps = [synth.make_problem(H=h, W=w, L_l=9, L_h=3, L_s=5, d=4, blur_size=5, blur_sigma=1.0, K=1, S=2,
                             lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=200 + i)
          for i, (h, w) in enumerate(sizes)]
    fs = [Fusion.from_problem(p, dtype="f32", wdtype="bf16") for p in ps]
    yl = [torch.tensor(p.Yl, dtype=torch.float32, device="cuda") for p in ps]
    yh = [torch.tensor(p.Yh, dtype=torch.float32, device="cuda") for p in ps]
    for f, h in zip(fs, yh):
        f.weights(h)
    return ps, fs, yl, yh


def test_batch_run_host_matches_device_path():
    ps, fs, yl, yh = _batch()
    b = FusionBatch(fs)
    Xs, Zs = b.solve(yl, yh, 14, want_X=True, want_Z=True)
    b.sync()
    hyl = [torch.tensor(p.Yl, dtype=torch.float32).pin_memory() for p in ps]
    hyh = [torch.tensor(p.Yh, dtype=torch.float32).pin_memory() for p in ps]
    for _ in range(2):
        Xh, Zh = b.run_host(hyl, hyh, 14, want_X=True, want_Z=True)
        for X, Z, x, z in zip(Xs, Zs, Xh, Zh):
            assert torch.equal(X.cpu(), x) and torch.equal(Z.cpu(), z)
    # an explicit guide (here Y_h itself) gives the same
    _, Zg = b.run_host(hyl, hyh, 14, want_X=False, want_Z=True, guides=hyh)
    for Z, z in zip(Zs, Zg):
        assert torch.equal(Z.cpu(), z)
    b.close()


def test_batch_long_solve_chunks_and_stale_state():
    # 270 batched iterations (a 256-iteration loop and a 14-iteration one) equal direct launches;
    # a second solve on the same contexts (their state left from the first) gives the same bits
    ps, fs, yl, yh = _batch(3)
    b = FusionBatch(fs)
    Xg, _ = b.solve(yl, yh, 270)
    b.sync()
    Xg = [x.clone() for x in Xg]
    Xg2, _ = b.solve(yl, yh, 270)
    b.sync()
    b.set_option(FUSE_OPT_GRAPH, 0)
    Xd, _ = b.solve(yl, yh, 270)
    b.sync()
    for a, c, d in zip(Xg, Xg2, Xd):
        assert torch.equal(a, c) and torch.equal(a, d)
    b.close()
