"""bench.py's host-side formulas: the algorithmic bytes of a latent launch counted element by
element on small shapes, the weak-scaling value, and the stored DRAM traffic of the latent
captures (reported only for the sources it was taken on)."""
import pathlib
import sys

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))
import bench  # noqa: E402
from paper_2210_04184_gb300 import synth  # noqa: E402


def _count(p, esz, wsz, half, ssz):
    """Bytes a latent launch must move, counted per stored array: every kept (tau, k) plane of the
    state read and written, the kept offsets' weights, X once, and the 2 planes per tau1 row."""
    n = p.H * p.W
    offs = [(a, b) for a in range(-p.S, p.S + 1) for b in range(-p.S, p.S + 1) if (a, b) != (0, 0)]
    kept = [t for t in offs if not half or t[0] > 0 or (t[0] == 0 and t[1] > 0)]
    rows = sorted({t[0] for t in kept})
    total = 0
    for _ in kept:
        total += (2 * p.K + 1) ** 2 * p.L_s * n * 2 * ssz        # state read + write
        total += n * wsz                                         # that offset's weights
    total += p.L_s * n * esz                                     # X
    total += len(rows) * 2 * p.L_s * n * esz                     # A and V planes per tau1 row
    return total


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("esz,wsz,ssz", [(4, 2, 4), (4, 4, 4), (8, 8, 8), (4, 2, 2)])
def test_latent_bytes_matches_an_explicit_count(half, esz, wsz, ssz):
    p = synth.make_problem(H=16, W=24, L_l=5, L_h=2, L_s=3, d=4, blur_size=3, K=1, S=2, seed=1)
    assert bench.latent_bytes(p, esz, wsz, half=half, ssz=ssz) == _count(p, esz, wsz, half, ssz)


def test_benchmark_latent_bytes():
    # hsms_256: 6.34 GB per launch with the FP32 state and BF16 weights, half window
    p, _ = synth.workload("hsms_256")
    assert bench.latent_bytes(p, 4, 2) == 6341787648


def test_job_value_and_single_rank_max():
    assert bench.job_value(10.0, 4, 2.0) == 20.0
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_stored_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    # the stored DRAM traffic scales with the pixel count while the latent sources match the
    # digest recorded with the capture, and is withheld (None) once they differ
    t = bench.LATENT_TRAFFIC["batch"]
    monkeypatch.setattr(bench, "_sources_digest", lambda: t["sources"])
    a = bench.latent_traffic("batch", 1000)
    assert a == pytest.approx(t["bytes_per_pixel"] * 1000)
    assert bench.latent_traffic("batch", 2000) == pytest.approx(2 * a)
    monkeypatch.setattr(bench, "_sources_digest", lambda: "0" * 16)
    assert bench.latent_traffic("batch", 1000) is None
    assert bench.latent_traffic("no such kernel", 1000) is None


def test_stored_traffic_is_close_to_the_algorithmic_bytes():
    # each capture moved close to the algorithmic bytes of its workload (no wasted re-reads)
    p, _ = synth.workload("hsms_256")
    alg = bench.latent_bytes(p, 4, 2) / (p.H * p.W)
    assert 0.9 <= bench.LATENT_TRAFFIC["hsms"]["bytes_per_pixel"] / alg <= 1.05
    ps = synth.batch_workload(8)
    alg8 = sum(bench.latent_bytes(q, 4, 2) for q in ps) / sum(q.H * q.W for q in ps)
    assert 0.95 <= bench.LATENT_TRAFFIC["batch"]["bytes_per_pixel"] / alg8 <= 1.05
