"""Precision study: the conditioning the iterate type has to carry (fuse_conditioning) against
independent FP64 computations of the same systems, on the workloads' parameters."""
import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import nlpr  # noqa: E402
from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300.fuse import Fusion, fuse_conditioning  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


@pytest.mark.parametrize("name", ["pansharpen_128", "hsms_128", "unrolled_256"])
def test_conditioning_matches_fp64_reference(name):
    p, meta = synth.workload(name)
    f = Fusion.from_problem(p, dtype=meta["dtype"], wdtype=meta["wdtype"])
    cA, cP1, cF = fuse_conditioning(f.ctx)
    den = nlpr.x_denominator(p.H, p.W, p.blur, p.K, p.S)        # eigenvalues of A (eq. inv)
    assert abs(cA - den.max() / den.min()) <= 1e-9 * cA
    L = p.E.shape[0]
    assert abs(cP1 - np.linalg.cond(p.E @ p.E.T + p.rho * np.eye(L))) <= 1e-9 * cP1
    G = p.E @ p.R
    assert abs(cF - np.linalg.cond(np.eye(L) + p.lam1 / p.rho * G @ G.T)) <= 1e-7 * cF
    # every system is far from the FP32 limit (1/eps = 1.7e7)
    assert max(cA, cP1, cF) < 1e6
