"""GPU parity of the register-resident DFT solve of the X system (FUSE_OPT_FFT_IMPL = 1, one warp
per line, sides N = 32 P) through the C-ABI.

Every P the form supports that the other GPU tests do not already reach through the default
path (they cover 1, 2, 3, 4, 8) appears along a row or a column here, with H != W so that a swapped
axis or a transposed factor fails.  Against the FP64 oracle (Sec. IV-A eqs.
x_linear_system_main and inv inside whole ADMM iterations): FP32 within 1e-5 relative
Frobenius error, FP64 within 1e-11.  Against the shared-memory Stockham form on the same
inputs: the same DFT up to rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300.fuse import (Fusion, FuseError, FUSE_OPT_FFT_IMPL)  # noqa: E402
from test_gpu_parity import gpu_solve, oracle_solve, rel, small  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


# (H, W): P along columns (H / 32) and rows (W / 32)
SHAPES = [(160, 192), (320, 96), (64, 384), (512, 64), (96, 320)]


@pytest.mark.parametrize("H,W", SHAPES)
def test_register_fft_fp32_matches_oracle(H, W):
    p = small(H=H, W=W, L_l=5, L_h=2, L_s=3, K=1, S=1, blur_size=5)
    g = gpu_solve(p, 3, opts=[(FUSE_OPT_FFT_IMPL, 1)])
    assert g["f"].get_option(FUSE_OPT_FFT_IMPL) == 1
    Xo, _, _ = oracle_solve(p, 3)
    assert rel(g["X"], Xo) <= 1e-5
    Zo = np.einsum("chw,cl->lhw", Xo, p.E)
    assert rel(g["Z"], Zo) <= 1e-5


@pytest.mark.parametrize("H,W", [(160, 192), (96, 320)])
def test_register_fft_fp64_matches_oracle(H, W):
    p = small(H=H, W=W, L_l=5, L_h=2, L_s=3, K=1, S=1, blur_size=5)
    g = gpu_solve(p, 3, dtype="f64", wdtype="f64", opts=[(FUSE_OPT_FFT_IMPL, 1)])
    Xo, _, _ = oracle_solve(p, 3)
    assert rel(g["X"], Xo) <= 1e-11


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("f64", 1e-13)])
def test_register_fft_equals_stockham(dtype, tol):
    # both forms on the same inputs: the same DFT solve up to rounding (P = 16 rows, 12 columns,
    # odd L_s: the last pair carries one band)
    p = small(H=384, W=512, L_l=6, L_h=2, L_s=5, K=1, S=1, blur_size=5)
    wd = "f64" if dtype == "f64" else "f32"
    a = gpu_solve(p, 2, dtype=dtype, wdtype=wd, opts=[(FUSE_OPT_FFT_IMPL, 1)])
    b = gpu_solve(p, 2, dtype=dtype, wdtype=wd, opts=[(FUSE_OPT_FFT_IMPL, 0)])
    assert rel(a["X"], b["X"]) <= tol


def test_fft_form_option():
    ok = Fusion.from_problem(small(H=64, W=96), dtype="f32", wdtype="f32")
    assert ok.get_option(FUSE_OPT_FFT_IMPL) == 1          # default where the sides allow it
    ok.set_option(FUSE_OPT_FFT_IMPL, 0)
    assert ok.get_option(FUSE_OPT_FFT_IMPL) == 0
    other = Fusion.from_problem(small(H=40, W=40), dtype="f32", wdtype="f32")
    assert other.get_option(FUSE_OPT_FFT_IMPL) == 0       # 40 = 32 P has no integer P
    with pytest.raises(FuseError):
        other.set_option(FUSE_OPT_FFT_IMPL, 1)


def test_switching_the_form_recaptures_the_loop():
    # a solve, a switch of the DFT form on the same context, another solve: each equals a fresh
    # context of that form bit for bit (the captured iteration loop is dropped on the switch)
    p = small(H=96, W=64, L_l=5, L_h=2, L_s=3, K=1, S=1, blur_size=5)
    yl = torch.tensor(p.Yl, dtype=torch.float32, device="cuda")
    yh = torch.tensor(p.Yh, dtype=torch.float32, device="cuda")

    def solve(f):
        X, _ = f.solve(yl, yh, 4)
        f.sync()
        return X.clone()

    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    f.weights(yh)
    a1 = solve(f)
    f.set_option(FUSE_OPT_FFT_IMPL, 0)
    a0 = solve(f)
    for form, got in ((1, a1), (0, a0)):
        g = Fusion.from_problem(p, dtype="f32", wdtype="f32")
        g.set_option(FUSE_OPT_FFT_IMPL, form)
        g.weights(yh)
        assert torch.equal(solve(g), got)
    assert not torch.equal(a0, a1)          # the two forms round differently
