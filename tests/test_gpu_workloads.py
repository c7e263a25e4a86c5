"""Parity at the workloads' own sizes and launch configurations (bench.py's defaults).

- pansharpening 128x128x4, FP64, 50 iterations: whole run against the oracle (1e-11);
- unrolled-forward workload 256x256x31 -> L_s 8, 20 iterations: whole run (1e-5);
- HS+MS 256x256x93 -> L_s 20 (the benchmark workload): the first three iterations against the
  oracle (the third is the first with a nonzero latent state), and after the full 100
  iterations the invariant |Sigma'| <= mu on sampled state entries;
- HS+PAN parameters (128 bands -> 20, 11x11 blur, K = 2, S = 5) on a 64x64 crop: 8 iterations.
- at the workloads' own iteration counts against the oracle, element by element: HS+MS at its
  full size for all 100 iterations (X, Z and sampled latent state), and the HS+PAN parameters on
  a 128 x 128 crop for all 200 iterations (its full size needs 252 GB of oracle state).
"""
import os

import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300.fuse import Fusion  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def _host_gib():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu(p, iters, dtype, wdtype, omega=None):
    td = torch.float64 if dtype == "f64" else torch.float32
    f = Fusion.from_problem(p, dtype=dtype, wdtype=wdtype)
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    if omega is None:
        f.weights(yh)
    else:
        f.set_weights(torch.tensor(omega, dtype=f.wtdtype, device="cuda"))
    X, Z = f.solve(yl, yh, iters, want_Z=True)
    f.sync()
    return X.double().cpu().numpy(), Z.double().cpu().numpy(), f


def _oracle(p, iters, omega):
    X, st, _ = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S,
                         p.lam1, p.lam2, p.rho, omega, iters, fast=True, inplace=True)
    return nlpr.to_lhw(X)


def test_pansharpen_fp64_full_size():
    p, meta = synth.workload("pansharpen_128")
    assert meta["dtype"] == "f64"
    X, Z, _ = _gpu(p, p.iters, "f64", "f64")
    from oracle import cloops
    om = cloops.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    Xo = _oracle(p, p.iters, om)
    assert rel(X, Xo) <= 1e-11
    assert rel(Z, np.einsum("chw,cl->lhw", Xo, p.E)) <= 1e-11


def test_unrolled_forward_full_size():
    p, meta = synth.workload("unrolled_256")
    X, Z, _ = _gpu(p, p.iters, "f32", "f32")
    from oracle import cloops
    om = cloops.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    Xo = _oracle(p, p.iters, om)
    assert rel(X, Xo) <= 1e-5


def test_hsms_full_size_first_iterations():
    p, meta = synth.workload("hsms_256")
    need = 2 * 48 * 25 * 20 * 256 * 256 * 8 / 2 ** 30 + 4          # Q and Sigma in FP64
    if _host_gib() < need * 1.2:
        pytest.skip(f"host has {_host_gib():.0f} GiB available, the oracle needs {need:.0f}")
    from oracle import cloops
    om = nlpr.round_bf16(cloops.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h))
    X, _, _ = _gpu(p, 3, "f32", "bf16", omega=om)
    Xo = _oracle(p, 3, om)
    assert rel(X, Xo) <= 1e-5


def test_hsms_full_size_latent_invariant():
    # After the benchmark's 100 iterations every latent entry satisfies |Sigma'| <= mu
    # (Sigma' = -clamp(v, -mu, mu), eqs. Qj_main and dualvar3_main); checked on a sample.
    p, meta = synth.workload("hsms_256")
    X, Z, f = _gpu(p, p.iters, "f32", "bf16")
    assert np.all(np.isfinite(X))
    st = f.get_state()
    om = f.get_weights().double().cpu().numpy()
    n, Ls = p.H * p.W, p.L_s
    img = n * Ls
    kept = [t for t, tau in enumerate(nlpr.search_offsets(p.S)) if tau[0] > 0 or (tau[0] == 0 and tau[1] > 0)]
    poffs = nlpr.patch_offsets(p.K)
    sig = st[5 * img * 4:(5 * img + len(kept) * len(poffs) * img) * 4].view(torch.float32)
    sig = sig.reshape(len(kept), len(poffs), Ls, p.H, p.W)
    rng = np.random.default_rng(5)
    coef = np.float32(p.lam2 / p.rho)
    nz = 0
    for _ in range(4000):
        j = int(rng.integers(len(kept))); kk = int(rng.integers(len(poffs)))
        c = int(rng.integers(Ls)); y = int(rng.integers(p.H)); x = int(rng.integers(p.W))
        k = poffs[kk]
        mu = coef * np.float32(om[kept[j], (y + k[0]) % p.H, (x + k[1]) % p.W])
        s = float(sig[j, kk, c, y, x].item())
        assert abs(s) <= mu * (1 + 1e-6)
        nz += s != 0.0
    assert nz > 0


def test_hspan_parameters_on_crop():
    p = synth.make_problem(H=64, W=64, L_l=128, L_h=1, L_s=20, d=4, blur_size=11, blur_sigma=2.0,
                           snr_l=30.0, snr_h=30.0, K=2, S=5, kind="hspan", seed=synth.SEED_BASE + 2)
    X, _, _ = _gpu(p, 8, "f32", "f32")
    from oracle import cloops
    om = cloops.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h)
    Xo = _oracle(p, 8, om)
    assert rel(X, Xo) <= 1e-5


def test_hspan_full_size_sampled():
    # HS+PAN at its full size (512 x 512, 128 bands -> L_s 20, 11x11 blur, K = 2, S = 5,
    # 120 offsets).  The oracle cannot hold its latent state (252 GB in FP64), so it computes
    # the first two iterations' images in full (X_2 only needs the pixel updates of iteration 1:
    # X_1 = 0 leaves the latent state at 0) and the latent state after iteration 2 entry by entry
    # on a sample: Sigma'(tau, k, c, m) = -clamp(X_2(m) - X_2(m - tau), lambda2 omega_tau(m+k)/rho).
    p, meta = synth.workload("hspan_512")
    X, _, f = _gpu(p, 2, meta["dtype"], meta["wdtype"])
    Yl, Yh = nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh)
    dummy = np.zeros((1, 1, 1))
    su = nlpr.setup(Yl, Yh, p.blur, p.d, p.R, p.E, p.K, p.S, p.lam1, p.lam2, p.rho, dummy)
    st = nlpr.State(*(np.zeros((p.H, p.W, p.L_s)) for _ in range(4)), Q=np.zeros(1), Sig=np.zeros(1))
    X1 = np.zeros((p.H, p.W, p.L_s))
    P1, BX = nlpr.update_p1(X1, st, su)
    P2 = nlpr.update_p2(X1, st, su)
    L1, L2 = -(BX - P1), -(X1 - P2)
    X2 = nlpr.solve_x(nlpr.blur_t(P1 + L1, p.blur) + P2 + L2, su.denom)
    assert rel(X, nlpr.to_lhw(X2)) <= 1e-5
    om = f.get_weights().double().cpu().numpy()
    state = f.get_state()
    n, Ls = p.H * p.W, p.L_s
    img = n * Ls
    offs = nlpr.search_offsets(p.S)
    kept = [t for t, tau in enumerate(offs) if tau[0] > 0 or (tau[0] == 0 and tau[1] > 0)]
    poffs = nlpr.patch_offsets(p.K)
    sig = state[5 * img * 4:(5 * img + len(kept) * len(poffs) * img) * 4].view(torch.float32)
    sig = sig.reshape(len(kept), len(poffs), Ls, p.H, p.W)
    rng = np.random.default_rng(6)
    coef = p.lam2 / p.rho
    # the clamp is 1-Lipschitz, so an entry differs by at most the FP32 error of its difference
    # of X_2 values (absolute, X ~ 1) plus the rounding of the threshold
    xs = np.abs(X2).max()
    nz = 0
    for _ in range(3000):
        j = int(rng.integers(len(kept))); kk = int(rng.integers(len(poffs)))
        c = int(rng.integers(Ls)); y = int(rng.integers(p.H)); x = int(rng.integers(p.W))
        tau, k = offs[kept[j]], poffs[kk]
        mu = coef * om[kept[j], (y + k[0]) % p.H, (x + k[1]) % p.W]
        v = X2[y, x, c] - X2[(y - tau[0]) % p.H, (x - tau[1]) % p.W, c]
        want = -min(max(v, -mu), mu)
        got = float(sig[j, kk, c, y, x].item())
        assert abs(got - want) <= 1e-6 * mu + 5e-6 * xs, (got, want, mu)
        nz += want != 0.0
    assert nz > 0


def test_hspan_full_size_fp32_vs_fp64_and_invariant():
    # the benchmark's 200 iterations at full size: FP32 (BF16 weights) against the FP64 GPU form
    # within the equal-error bound, and |Sigma'| <= mu on sampled state entries
    p, meta = synth.workload("hspan_512")
    X32, Z32, f = _gpu(p, p.iters, meta["dtype"], meta["wdtype"])
    assert np.all(np.isfinite(Z32))
    st = f.get_state()
    om = f.get_weights().double().cpu().numpy()
    n, Ls = p.H * p.W, p.L_s
    img = n * Ls
    offs = nlpr.search_offsets(p.S)
    kept = [t for t, tau in enumerate(offs) if tau[0] > 0 or (tau[0] == 0 and tau[1] > 0)]
    poffs = nlpr.patch_offsets(p.K)
    sig = st[5 * img * 4:(5 * img + len(kept) * len(poffs) * img) * 4].view(torch.float32)
    sig = sig.reshape(len(kept), len(poffs), Ls, p.H, p.W)
    rng = np.random.default_rng(7)
    coef = np.float32(p.lam2 / p.rho)
    for _ in range(3000):
        j = int(rng.integers(len(kept))); kk = int(rng.integers(len(poffs)))
        c = int(rng.integers(Ls)); y = int(rng.integers(p.H)); x = int(rng.integers(p.W))
        k = poffs[kk]
        mu = coef * np.float32(om[kept[j], (y + k[0]) % p.H, (x + k[1]) % p.W])
        assert abs(float(sig[j, kk, c, y, x].item())) <= mu * (1 + 1e-6)
    del st, sig, f
    torch.cuda.empty_cache()
    X64, Z64, _ = _gpu(p, p.iters, "f64", "f64")
    assert rel(Z32, Z64) <= 1e-4


def test_hspan_full_size_fixed_point_state():
    # the 16-bit fixed-point state on the largest workload (512 x 512, 120 offsets, 200
    # iterations): Z within the equal-error bound of the FP64 GPU form
    from paper_2210_04184_gb300.fuse import FUSE_OPT_STATE_FORMAT
    p, meta = synth.workload("hspan_512")
    f = Fusion.from_problem(p, dtype="f32", wdtype="bf16")
    f.set_option(FUSE_OPT_STATE_FORMAT, 1)
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")
    f.weights(yh)
    _, Z = f.solve(yl, yh, p.iters, want_X=False, want_Z=True)
    f.sync()
    Zq = Z.double().cpu().numpy()
    f.close()
    del Z
    torch.cuda.empty_cache()
    _, Z64, _ = _gpu(p, p.iters, "f64", "f64")
    assert rel(Zq, Z64) <= 1e-4


def _kept_offsets(S):
    return [t for t, tau in enumerate(nlpr.search_offsets(S)) if tau[0] > 0 or (tau[0] == 0 and tau[1] > 0)]


def _full_run_parity(p, iters, seed):
    """FP32 iterates with BF16 weights (the oracle's FP64 weights rounded to BF16 and given to both
    sides) after `iters` iterations from zero: X and Z element by element within 1e-5 relative
    Frobenius of the FP64 oracle, and 4000 sampled entries of the latent state against the
    oracle's Sigma (stored re-indexed by the source pixel on the GPU:
    Sig'[tau][k][c][m] = Sigma_{tau k}(m + k))."""
    from oracle import cloops
    om = nlpr.round_bf16(cloops.weights(nlpr.to_hwl(p.Yh), p.K, p.S, p.h))
    X, Z, f = _gpu(p, iters, "f32", "bf16", omega=om)
    st = f.get_state().cpu()
    f.close()
    torch.cuda.empty_cache()
    Xo, sto, _ = nlpr.admm(nlpr.to_hwl(p.Yl), nlpr.to_hwl(p.Yh), p.blur, p.d, p.R, p.E, p.K, p.S,
                           p.lam1, p.lam2, p.rho, om, iters, fast=True, inplace=True)
    Xo = nlpr.to_lhw(Xo)
    assert rel(X, Xo) <= 1e-5
    assert rel(Z, np.einsum("chw,cl->lhw", Xo, p.E)) <= 1e-5
    n, Ls = p.H * p.W, p.L_s
    img = n * Ls
    kept = _kept_offsets(p.S)
    poffs = nlpr.patch_offsets(p.K)
    sig = st[5 * img * 4:(5 * img + len(kept) * len(poffs) * img) * 4].view(torch.float32)
    sig = sig.reshape(len(kept), len(poffs), Ls, p.H, p.W).numpy()
    rng = np.random.default_rng(seed)
    scale = float(np.abs(sto.Sig).max())
    nz = 0
    for _ in range(4000):
        j = int(rng.integers(len(kept))); kk = int(rng.integers(len(poffs)))
        c = int(rng.integers(Ls)); y = int(rng.integers(p.H)); x = int(rng.integers(p.W))
        k = poffs[kk]
        want = sto.Sig[kept[j], kk, (y + k[0]) % p.H, (x + k[1]) % p.W, c]
        got = float(sig[j, kk, c, y, x])
        # each entry is -clamp(v, -mu, mu) with v a difference of X values: 1-Lipschitz in X
        assert abs(got - want) <= 1e-5 * scale + 1e-5 * float(np.abs(Xo).max()), (got, want)
        nz += want != 0.0
    assert nz > 0


def test_hsms_full_size_all_iterations():
    # the benchmarked single-problem workload at its size and its 100 iterations
    p, meta = synth.workload("hsms_256")
    need = 2 * 48 * 25 * 20 * 256 * 256 * 8 / 2 ** 30 + 6
    if _host_gib() < need * 1.2:
        pytest.skip(f"host has {_host_gib():.0f} GiB available, the oracle needs {need:.0f}")
    _full_run_parity(p, p.iters, 11)


def test_hspan_crop_all_iterations():
    # every HS+PAN parameter (128 bands -> L_s 20, 11x11 blur sigma 2, 30 dB, K = 2, S = 5,
    # 120 offsets) and its 200 iterations on a 128 x 128 crop, with the workload's BF16 weights
    spec = dict(synth.WORKLOADS["hspan_512"])
    for k in ("dtype", "wdtype", "cfg", "H", "W"):
        spec.pop(k)
    p = synth.make_problem(H=128, W=128, seed=synth.SEED_BASE + 2, **spec)
    assert p.iters == 200 and p.S == 5 and p.K == 2 and p.L_s == 20
    need = 2 * 120 * 25 * 20 * 128 * 128 * 8 / 2 ** 30 + 4
    if _host_gib() < need * 1.2:
        pytest.skip(f"host has {_host_gib():.0f} GiB available, the oracle needs {need:.0f}")
    _full_run_parity(p, p.iters, 12)
