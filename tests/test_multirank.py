"""Host logic of multi-process runs (world size 2, gloo on CPU): every rank gets its own seeded
problem (weak scaling, no data-path collective), the timing is the maximum over ranks, and the
whole-job value counts every rank's units over that time."""
import os
import pathlib
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = pathlib.Path(__file__).resolve().parents[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slow = bench.max_over_ranks(1.0 + 2.0 * rank, dist, device="cpu")
        p, meta = bench._workload("unrolled_256", rank, 2)
        val = bench.job_value(10.0, world, slow)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([slow, val, meta["seed"], float(p.Yh[0, 0, 0]), float(p.Yl[0, 0, 0])]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_timing_and_distinct_problems(tmp_path):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(timeout=300)
        assert q.exitcode == 0
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 3.0                 # the slowest rank's time on both
    assert r0[1] == r1[1] == 10.0 * 2 / 3.0      # units of both ranks over that time
    assert r0[2] != r1[2]                        # a different seeded problem per rank
    assert r0[3] != r1[3] and r0[4] != r1[4]
