"""fuse_phi_static: the regulariser value without any device allocation, for callers that may
not allocate (under a host-owned GPU memory budget, or where cudaMalloc's implicit device
synchronisation is not affordable).  Checked through the C-ABI against fuse_objective's
regulariser term on two calls in a row (the second call finds the previous call's partial sums
in the shared array), and against the FP64 oracle's phi (eq. reg1) evaluated on the same X and
weights copied to the host."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300 import fuse  # noqa: E402
from paper_2210_04184_gb300.fuse import Fusion, FuseError  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


@pytest.mark.parametrize("dtype,wdtype", [("f32", "f32"), ("f32", "bf16"), ("f64", "f64")])
def test_phi_static_matches_objective_twice(dtype, wdtype):
    p = synth.make_problem(H=48, W=64, L_l=8, L_h=3, L_s=4, d=4, blur_size=9, blur_sigma=1.7, K=2, S=3,
                           lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=21)
    td = torch.float64 if dtype == "f64" else torch.float32
    f = Fusion.from_problem(p, dtype=dtype, wdtype=wdtype)
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    f.weights(yh)
    X, _ = f.solve(yl, yh, 12)
    obj = f.objective(yl, yh)                 # existing entry point: obj[2] = lambda2 * phi(X)
    om = f.get_weights()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        fuse.fuse_phi_static(X.data_ptr(), om.data_ptr(), p.H, p.W, p.L_s, p.K, p.S,
                             fuse.DTYPES[dtype], fuse.DTYPES[wdtype], out.data_ptr(), stream)
        torch.cuda.synchronize()
        phi = float(out.item())
        assert abs(p.lam2 * phi - obj[2]) <= 1e-5 * abs(obj[2])
    # the oracle's phi on the GPU's own X and weights (FP32: per-pixel sums in FP32, 1e-5; FP64: 1e-11)
    ref = nlpr.nlpr(nlpr.to_hwl(X.double().cpu().numpy()), om.double().cpu().numpy(), p.K, p.S)
    assert abs(phi - ref) <= (1e-11 if dtype == "f64" else 1e-5) * abs(ref)
    f.close()


def test_phi_static_rejects_sizes_beyond_its_array():
    # ceil(H*W/256) * |W| partial sums must fit in 2^18: 1024 x 1024 with S = 5 (120 offsets)
    # needs 491520 and is refused before any work is issued.
    X = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(FuseError) as e:
        fuse.fuse_phi_static(X.data_ptr(), X.data_ptr(), 1024, 1024, 4, 1, 5, fuse.FUSE_F32, fuse.FUSE_F32,
                             out.data_ptr(), 0)
    assert e.value.status == fuse.FUSE_EUNSUPPORTED
