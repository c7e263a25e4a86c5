#!/usr/bin/env python3
"""Benchmark of the NLPR fusion ADMM on GB300 (prints one JSON line on rank 0).

A step is one pass of the whole hot path over one synthetic problem: guide weights
(eq. wts), `iters` ADMM iterations (Sec. IV) and the output Z = X E.  The default workload
is HS+MS fusion at 256 x 256 x 93 bands, subspace L_s = 20, 5x5 patches, 7x7 search window,
BF16 weights, FP32 iterates, 100 iterations.

Metric: megapixel-band-iterations per second, (H W / 1e6) L_s iters / seconds, summed over
ranks (each rank solves its own independent problem: weak scaling, no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import pathlib
import statistics
import subprocess
import sys
import threading
import time

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

METRIC = "ADMM throughput (megapixel*band*iter/s)"

# nominal HBM3e bandwidth of one GB300 (context only; the roofline divides by the measured copy)
NOMINAL_HBM_GBS = 7900.0

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one latent-pass launch, from an
# ncu capture of the 128x128 case of the same workload (the same kernel and launch shape), per
# pixel; scaled to the workload by its pixel count (the traffic is proportional to it).  Must be
# re-measured whenever the latent kernel changes.
LATENT_TRAFFIC_PER_PIXEL = {"hsms": (788.702720e6 + 738.255872e6) / (128 * 128)}
UNIT = "Mpx*band*iter/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hsms_256")
    ap.add_argument("--iters", type=int, default=None, help="override the workload's iteration count")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-vs-FP32 comparison")
    ap.add_argument("--no-grad", action="store_true", help="skip the reverse-pass measurement")
    ap.add_argument("--grad-only", action="store_true", help="only the reverse-pass measurement")
    ap.add_argument("--grad-workload", default="unrolled_256", help="workload of the reverse-pass measurement")
    ap.add_argument("--no-fixed", action="store_true", help="skip the fixed-point state measurement")
    ap.add_argument("--no-sb", action="store_true", help="skip the S B-in-X update measurement")
    ap.add_argument("--fixed-state", action="store_true",
                    help="run the main measurement with the 16-bit fixed-point latent state")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    return ap.parse_args()


def _peaks():
    try:
        return json.loads((ROOT / "MEASURED_PEAKS.json").read_text())
    except Exception:
        return {}


def _workload(name, rank, iters_override):
    from paper_2210_04184_gb300 import synth
    spec = synth.WORKLOADS[name]
    p, meta = synth.workload(name, seed=synth.SEED_BASE + spec["cfg"] + 7919 * rank)
    if iters_override:
        p.iters = iters_override
    return p, meta


def _config(p, meta, name, n_gpus):
    return {
        "workload": name,
        "H": p.H, "W": p.W, "bands": p.L_l, "L_h": p.L_h, "L_s": p.L_s, "ratio": p.d,
        "patch": f"{2 * p.K + 1}x{2 * p.K + 1}", "search": f"{2 * p.S + 1}x{2 * p.S + 1}",
        "offsets": (2 * p.S + 1) ** 2 - 1, "iters": p.iters, "weights": meta["wdtype"],
        "global_batch": n_gpus, "parallelism": f"independent problems x{n_gpus}",
        "l2": "latent state per problem exceeds L2 (no flush needed)",
        "latent_state": "half window (one offset of each +-tau pair)",
    }


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of a host float over all ranks (the max-over-ranks timing of a weak-
    scaling run: every rank solves its own problems, and no collective touches the data path)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def latent_bytes(p, esz, wsz, half=True, ssz=None):
    """Algorithmic bytes of one latent-pass launch: state read + write over the kept offsets
    (half of the window in half-window mode; ssz bytes per stored entry, default esz), their
    weights, X, and the adjoint planes."""
    n = p.H * p.W
    nW = (2 * p.S + 1) ** 2 - 1
    nK = nW // 2 if half else nW
    rows = p.S + 1 if half else 2 * p.S + 1
    nP = (2 * p.K + 1) ** 2
    ssz = ssz or esz
    return (2 * nK * nP * p.L_s * n * ssz + nK * n * wsz + p.L_s * n * esz
            + 2 * rows * p.L_s * n * esz)


def cpu_baseline(p, target_s=15.0):
    """The FP64 oracle timed on the host cores on a bounded crop of the same workload
    (same bands, subspace, patch and window; a 48 x 48 image; weights plus n iterations,
    n sized from a one-iteration probe so the sample takes about target_s seconds)."""
    from oracle import nlpr
    from paper_2210_04184_gb300 import synth
    crop = 48
    q = synth.make_problem(H=crop, W=crop, L_l=p.L_l, L_h=p.L_h, L_s=p.L_s, d=p.d,
                           blur_size=p.blur.shape[0], blur_sigma=1.7, K=p.K, S=p.S, lam1=p.lam1,
                           lam2=p.lam2, rho=p.rho, h=p.h, seed=1, kind="hsms")
    Yl, Yh = nlpr.to_hwl(q.Yl), nlpr.to_hwl(q.Yh)

    def run(n):
        t0 = time.perf_counter()
        om = nlpr.weights(Yh, q.K, q.S, q.h)
        nlpr.admm(Yl, Yh, q.blur, q.d, q.R, q.E, q.K, q.S, q.lam1, q.lam2, q.rho, om, n, fast=True)
        return time.perf_counter() - t0

    run(1)                      # first touch of the oracle's arrays
    probe = run(1)
    n = int(max(1, min(100, target_s / max(probe, 1e-3))))
    dt = run(n)
    value = crop * crop / 1e6 * q.L_s * n / dt
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{crop}x{crop} crop, {q.L_l} bands, L_s={q.L_s}, K={q.K}, S={q.S}, "
                      f"weights + {n} iterations, FP64 NumPy + C/OpenMP loops, {dt:.1f}s"}


def run_reference(a, rank, world):
    if rank != 0:
        return
    if a.workload == "batch64":
        from paper_2210_04184_gb300 import synth
        p = synth.batch_workload(1)[0]
        meta = {"dtype": "f32", "wdtype": "bf16"}
    else:
        p, meta = _workload(a.workload, 0, a.iters)
    samples = []
    cb = None
    for i in range(a.warmup + a.steps):
        cb = cpu_baseline(p, target_s=8.0 if i >= a.warmup else 2.0)
        if i >= a.warmup:
            samples.append(cb["value"])
    value = statistics.median(samples)
    cb["value"] = value
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": _config(p, meta, a.workload, a.gpus), "cpu_baseline": cb,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def fp64_compare(p, meta, f32ctx, yl, yh, Z32):
    """The FP64 GPU form of the same workload (FP64 iterates and weights) against the FP32 form:
    iterations per second of each and the relative error of Z (FP32 with the run's weight type,
    and FP32 with FP32 weights) against the FP64 result, at the workload's iteration count."""
    import torch
    from paper_2210_04184_gb300.fuse import Fusion

    def timed(ctx, Yl, Yh, Zout):
        from paper_2210_04184_gb300.fuse import fuse_solve, fuse_weights, fuse_set_stream
        st = torch.cuda.current_stream()
        fuse_set_stream(ctx.ctx, st.cuda_stream)
        fuse_weights(ctx.ctx, Yh.data_ptr())
        fuse_solve(ctx.ctx, Yl.data_ptr(), Yh.data_ptr(), 2, 0, None, None)     # warm (graph capture)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fuse_solve(ctx.ctx, Yl.data_ptr(), Yh.data_ptr(), p.iters, 0, None, Zout.data_ptr())
        e1.record(st)
        ctx.sync()
        return p.iters / (e0.elapsed_time(e1) / 1e3)

    yl64, yh64 = yl.double(), yh.double()
    Z64 = torch.empty((p.L_l, p.H, p.W), dtype=torch.float64, device="cuda")
    f64 = Fusion.from_problem(p, dtype="f64", wdtype="f64")
    if "mask" in meta:
        f64.set_mask(meta["mask"])
    it64 = timed(f64, yl64, yh64, Z64)
    f64.close()
    it32 = timed(f32ctx, yl, yh, Z32)
    nz = torch.linalg.norm(Z64)
    err32 = float(torch.linalg.norm(Z32.double() - Z64) / nz)
    out = {"fp64_iters_per_s": it64, "fp32_iters_per_s": it32, "speedup": it32 / it64,
           "rel_err_Z_fp32_vs_fp64": err32, "fp32_weights": meta["wdtype"]}
    if meta["wdtype"] != "f32":
        fw = Fusion.from_problem(p, dtype="f32", wdtype="f32")
        if "mask" in meta:
            fw.set_mask(meta["mask"])
        Zw = torch.empty_like(Z32)
        timed(fw, yl, yh, Zw)
        fw.close()
        out["rel_err_Z_fp32_f32weights_vs_fp64"] = float(torch.linalg.norm(Zw.double() - Z64) / nz)
    out["equal_error_1e-4"] = out.get("rel_err_Z_fp32_f32weights_vs_fp64", err32) <= 1e-4
    return out, Z64


def fixed_point_bench(a, p, meta, yl, yh, Z64):
    """The same workload with the latent state stored in 16-bit fixed point relative to its
    threshold (FUSE_OPT_STATE_FORMAT = 1): throughput, the latent pass against the roofline
    (2-byte state entries), and the relative error of Z against the FP64 GPU run."""
    import torch
    from paper_2210_04184_gb300.fuse import (Fusion, FUSE_OPT_PROFILE, FUSE_K_LATENT, FUSE_OPT_STATE_FORMAT,
                                             fuse_solve, fuse_weights, fuse_set_stream)
    f = Fusion.from_problem(p, dtype=meta["dtype"], wdtype=meta["wdtype"])
    f.set_option(FUSE_OPT_STATE_FORMAT, 1)
    if "mask" in meta:
        f.set_mask(meta["mask"])
    st = torch.cuda.current_stream()
    fuse_set_stream(f.ctx, st.cuda_stream)
    fuse_weights(f.ctx, yh.data_ptr())
    tuned = f.autotune(yl, yh, iters=2)
    Z = torch.empty((p.L_l, p.H, p.W), dtype=yl.dtype, device="cuda")

    def step():
        fuse_weights(f.ctx, yh.data_ptr())
        fuse_solve(f.ctx, yl.data_ptr(), yh.data_ptr(), p.iters, 0, None, Z.data_ptr())

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    f.set_option(FUSE_OPT_PROFILE, 1)
    f.profile(FUSE_K_LATENT, reset=True)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat_ms, lat_n = f.profile(FUSE_K_LATENT)
    f.set_option(FUSE_OPT_PROFILE, 0)
    f.close()
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    wsz = {"bf16": 2, "f32": 4, "f64": 8}[meta["wdtype"]]
    lb = latent_bytes(p, 4, wsz, ssz=2)
    per = lat_ms / max(lat_n, 1)
    err = float(torch.linalg.norm(Z.double() - Z64) / torch.linalg.norm(Z64)) if Z64 is not None else None
    return {"state": "int16 fixed point relative to mu",
            "value": p.H * p.W / 1e6 * p.L_s * p.iters * a.steps / (ms / 1e3),
            "unit": UNIT, "ms_per_step": ms / a.steps, "launch_shapes": tuned,
            "roofline": {"bound": "hbm", "achieved": lb / (per / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": lb / (per / 1e3) / 1e9 / hbm, "kernel": "latent_tma_kernel<int16 state>",
                         "algorithmic_bytes_per_launch": lb, "avg_launch_ms": per, "launches": lat_n,
                         "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"},
            "rel_err_Z_vs_fp64": err, "equal_error_1e-4": err is not None and err <= 1e-4}


def sb_bench(a, p, meta, yl, yh, f0):
    """The same workload with the X update that keeps S B in the X system (FUSE_OPT_X_UPDATE = 1,
    alias-class solves in the column FFT pass): throughput, and the objective after the
    workload's iterations next to the paper's splitting (same objective, other iterates)."""
    import torch
    from paper_2210_04184_gb300.fuse import Fusion, FUSE_OPT_X_UPDATE, fuse_solve, fuse_weights, fuse_set_stream
    f = Fusion.from_problem(p, dtype=meta["dtype"], wdtype=meta["wdtype"])
    f.set_option(FUSE_OPT_X_UPDATE, 1)
    st = torch.cuda.current_stream()
    fuse_set_stream(f.ctx, st.cuda_stream)
    fuse_weights(f.ctx, yh.data_ptr())
    Z = torch.empty((p.L_l, p.H, p.W), dtype=yl.dtype, device="cuda")

    def step():
        fuse_weights(f.ctx, yh.data_ptr())
        fuse_solve(f.ctx, yl.data_ptr(), yh.data_ptr(), p.iters, 0, None, Z.data_ptr())

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    obj_sb = sum(f.objective(yl, yh)[:3])
    obj_paper = sum(f0.objective(yl, yh)[:3])
    f.close()
    return {"x_update": "S B kept in the X system (alias-class solves)",
            "value": p.H * p.W / 1e6 * p.L_s * p.iters * a.steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / a.steps, "iters": p.iters,
            "objective": obj_sb, "objective_paper_splitting": obj_paper}


def run_batch(a, rank, world, local_rank):
    """The batched uneven-tile workload: 64 problems of sizes 96..384, one launch per ADMM phase
    over all of them (FP32, BF16 weights), against per-problem sequential FP64 GPU solves."""
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2210_04184_gb300 import build as _build, synth
    from paper_2210_04184_gb300.fuse import (Fusion, FusionBatch, FUSE_OPT_PROFILE, FUSE_K_ALL,
                                             FUSE_K_LATENT, fuse_weights)
    _build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    nprob = 64
    ps = synth.batch_workload(nprob, seed=synth.SEED_BASE + 4 + 7919 * rank)
    iters = a.iters or ps[0].iters
    for p in ps:
        p.iters = iters
    fs = [Fusion.from_problem(p, dtype="f32", wdtype="bf16") for p in ps]
    yl = [torch.tensor(p.Yl, dtype=torch.float32, device="cuda") for p in ps]
    yh = [torch.tensor(p.Yh, dtype=torch.float32, device="cuda") for p in ps]
    batch = FusionBatch(fs)
    stream = torch.cuda.current_stream()
    for f, h in zip(fs, yh):
        fuse_weights(f.ctx, h.data_ptr())
    batch.autotune(yl, yh, iters=1)                # launch shapes only; results are unchanged

    def step():
        for f, h in zip(fs, yh):
            fuse_weights(f.ctx, h.data_ptr())
        return batch.solve(yl, yh, iters, want_X=False, want_Z=True)

    for _ in range(a.warmup):
        step()
    batch.sync()
    batch.set_option(FUSE_OPT_PROFILE, 1)
    batch.profile(FUSE_K_LATENT, reset=True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        _, Zs = step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    lat_ms, lat_n = batch.profile(FUSE_K_LATENT)
    _, launches = batch.profile(FUSE_K_ALL)
    batch.set_option(FUSE_OPT_PROFILE, 0)
    batch.sync()
    ms = max_over_ranks(ms, dist)
    px = sum(p.H * p.W for p in ps)
    Ls = ps[0].L_s
    units = px / 1e6 * Ls * iters * a.steps * world
    value = job_value(units / world, world, ms / 1e3)

    # end to end: pinned host inputs copied in, Z of every problem read back, each step
    e2e = None
    if not a.no_e2e:
        hyl = [torch.from_numpy(np.ascontiguousarray(p.Yl, dtype=np.float32)).pin_memory() for p in ps]
        hyh = [torch.from_numpy(np.ascontiguousarray(p.Yh, dtype=np.float32)).pin_memory() for p in ps]
        hz = [torch.empty((p.L_l, p.H, p.W), dtype=torch.float32).pin_memory() for p in ps]

        def e2e_step():
            dl = [h.to("cuda", non_blocking=True) for h in hyl]
            dh = [h.to("cuda", non_blocking=True) for h in hyh]
            for f, h in zip(fs, dh):
                fuse_weights(f.ctx, h.data_ptr())
            _, Zs2 = batch.solve(dl, dh, iters, want_X=False, want_Z=True)
            for z, hzz in zip(Zs2, hz):
                hzz.copy_(z, non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            e2e_step()
        dt = max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": units / dt, "unit": UNIT,
               "h2d_bytes_per_step": sum(h.numel() * 4 for h in hyl) + sum(h.numel() * 4 for h in hyh),
               "d2h_bytes_per_step": sum(h.numel() * 4 for h in hz)}

    # per-problem sequential FP64 GPU solves of the same problems
    seq = None
    if not a.no_fp64 and rank == 0:
        t64 = 0.0
        worst = 0.0
        for p, Z32 in zip(ps, Zs):
            f64 = Fusion.from_problem(p, dtype="f64", wdtype="f64")
            a64 = torch.tensor(p.Yl, dtype=torch.float64, device="cuda")
            b64 = torch.tensor(p.Yh, dtype=torch.float64, device="cuda")
            f64.weights(b64)
            f64.solve(a64, b64, 2, want_X=False)          # graph capture outside the timing
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            f64.weights(b64)
            _, Z64 = f64.solve(a64, b64, iters, want_X=False, want_Z=True)
            s1.record(stream)
            f64.sync()
            t64 += s0.elapsed_time(s1) / 1e3
            worst = max(worst, float(torch.linalg.norm(Z32.double() - Z64) / torch.linalg.norm(Z64)))
            f64.close()
        v64 = px / 1e6 * Ls * iters / t64
        seq = {"fp64_sequential_value": v64, "unit": UNIT, "speedup_fp32_batched": value / world / v64,
               "max_rel_err_Z_fp32_vs_fp64": worst, "equal_error_1e-4": worst <= 1e-4}

    if rank != 0:
        batch.close()
        if dist:
            dist.destroy_process_group()
        return
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    per_launch_ms = lat_ms / max(lat_n, 1)
    lb = sum(latent_bytes(p, 4, 2) for p in ps)
    achieved = lb / (per_launch_ms / 1e3) / 1e9
    sizes = sorted(set(p.H for p in ps))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch64", "problems": nprob, "sizes": sizes, "pixels": px, "bands": 31,
                   "L_h": 3, "L_s": Ls, "ratio": 4, "patch": "3x3", "search": "7x7", "iters": iters,
                   "weights": "bf16", "global_batch": nprob * world,
                   "parallelism": f"batched problems, independent batches x{world}",
                   "l2": "latent state exceeds L2 (no flush needed)",
                   "latent_state": "half window (one offset of each +-tau pair)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "latent_tma_batch_kernel", "algorithmic_bytes_per_launch": lb,
                     "avg_launch_ms": per_launch_ms, "launches": lat_n,
                     "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"},
        "gpu_launches": launches, "clocks": clk, "e2e": e2e, "fp64_sequential": seq,
    }
    print(json.dumps(out), flush=True)
    batch.close()
    if dist:
        dist.destroy_process_group()


def grad_bench(a, rank):
    """Forward with checkpoints and reverse pass (fuse_grad_forward / fuse_grad_backward) of the
    unrolled-forward workload (256 x 256, 31 bands, L_s 8, 3x3 patches, 3x3 search, 20
    iterations, FP32), loss <Wt, X_K> with a seeded Wt; against a plain fuse_solve of the same
    iterations and the oracle's FP64 reverse pass timed on a 32 x 32 crop."""
    import torch
    from oracle import grad as ograd, nlpr
    from paper_2210_04184_gb300 import synth
    from paper_2210_04184_gb300.fuse import Fusion, fuse_grad_bytes
    name = getattr(a, "grad_workload", "unrolled_256")
    p, meta = _workload(name, rank, a.iters if name != "unrolled_256" else None)
    td = torch.float32
    f = Fusion.from_problem(p, dtype=meta["dtype"], wdtype=meta["wdtype"])
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    Wt = torch.tensor(np.random.default_rng(17).standard_normal((p.L_s, p.H, p.W)), dtype=td, device="cuda")
    f.weights(yh)
    st = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for _ in range(max(3, a.warmup)):
        f.grad_forward(yl, yh, p.iters)
        f.grad_backward(Xbar=Wt)
        f.solve(yl, yh, p.iters, want_X=False)
    torch.cuda.synchronize()
    fwd, bwd, plain = [], [], []
    for _ in range(max(1, a.steps)):
        e0, e1, e2, e3, e4 = ev(), ev(), ev(), ev(), ev()
        e0.record(st)
        f.grad_forward(yl, yh, p.iters)
        e1.record(st)
        f.grad_backward(Xbar=Wt)            # includes the host read of the parameter sums
        e2.record(st)
        e3.record(st)
        f.solve(yl, yh, p.iters, want_X=False)
        e4.record(st)
        torch.cuda.synchronize()
        fwd.append(e0.elapsed_time(e1)); bwd.append(e1.elapsed_time(e2)); plain.append(e3.elapsed_time(e4))
    fm, bm, pm = statistics.median(fwd), statistics.median(bwd), statistics.median(plain)
    units = p.H * p.W / 1e6 * p.L_s * p.iters
    out = {"workload": name, "H": p.H, "W": p.W, "bands": p.L_l, "L_s": p.L_s,
           "patch": f"{2 * p.K + 1}x{2 * p.K + 1}", "search": f"{2 * p.S + 1}x{2 * p.S + 1}",
           "iters": p.iters, "dtype": "f32", "weights": meta["wdtype"],
           "ms_forward_with_tape": fm, "ms_backward": bm, "ms_plain_forward": pm,
           "value_forward_backward": units / ((fm + bm) / 1e3), "unit": UNIT,
           "backward_over_plain_forward": bm / pm, "workspace_bytes": fuse_grad_bytes(f.ctx, p.iters)}
    f.close()
    if rank == 0 and not a.no_cpu_baseline and name == "unrolled_256":
        # the oracle as it stands, the workload's 20 iterations on a square crop: 64 x 64, or
        # 128 x 128 when the 64 x 64 run took under 3 s (a sample of several seconds)
        spec = dict(synth.WORKLOADS["unrolled_256"])
        for k in ("dtype", "wdtype", "cfg", "iters", "H", "W"):
            spec.pop(k)
        iters = p.iters

        def run(crop):
            q = synth.make_problem(H=crop, W=crop, seed=1, **spec)
            om = nlpr.weights(nlpr.to_hwl(q.Yh), q.K, q.S, q.h)
            Wq = np.random.default_rng(0).standard_normal((crop, crop, q.L_s))
            t0 = time.perf_counter()
            ograd.unrolled_grad(nlpr.to_hwl(q.Yl), nlpr.to_hwl(q.Yh), q.blur, q.d, q.R, q.E, q.K, q.S, q.lam1,
                                q.lam2, q.rho, om, iters, lambda X: Wq)
            return time.perf_counter() - t0, q

        crop = 64
        dt, q = run(crop)
        if dt < 3.0:
            crop = 128
            dt, q = run(crop)
        out["cpu_baseline"] = {"value": crop * crop / 1e6 * q.L_s * iters / dt, "unit": UNIT, "cores": 1,
                               "kind": "oracle",
                               "sample": f"{crop}x{crop} crop, forward tape + reverse pass of {iters} "
                                         f"iterations, FP64 NumPy, {dt:.1f}s"}
    return out


def run_ours(a, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2210_04184_gb300 import build as _build
    from paper_2210_04184_gb300.fuse import Fusion, FUSE_OPT_PROFILE, FUSE_K_ALL, FUSE_K_LATENT
    _build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    p, meta = _workload(a.workload, rank, a.iters)
    td = torch.float64 if meta["dtype"] == "f64" else torch.float32
    esz = 8 if meta["dtype"] == "f64" else 4
    wsz = {"bf16": 2, "f32": 4, "f64": 8}[meta["wdtype"]]
    f = Fusion.from_problem(p, dtype=meta["dtype"], wdtype=meta["wdtype"])
    if a.fixed_state:
        from paper_2210_04184_gb300.fuse import FUSE_OPT_STATE_FORMAT
        f.set_option(FUSE_OPT_STATE_FORMAT, 1)
    if "mask" in meta:
        f.set_mask(meta["mask"])            # random sampling operator (inpainting workload)
    yl = torch.tensor(p.Yl, dtype=td, device="cuda")
    yh = torch.tensor(p.Yh, dtype=td, device="cuda")
    Z = torch.empty((p.L_l, p.H, p.W), dtype=td, device="cuda")
    stream = torch.cuda.current_stream()

    from paper_2210_04184_gb300.fuse import fuse_solve, fuse_weights, fuse_set_stream, fuse_conditioning
    fuse_set_stream(f.ctx, stream.cuda_stream)
    fuse_weights(f.ctx, yh.data_ptr())
    if a.no_autotune:
        from paper_2210_04184_gb300.fuse import (fuse_get_option, FUSE_OPT_LATENT_THREADS, FUSE_OPT_LATENT_STAGES,
                                                 FUSE_OPT_LATENT_BANDS, FUSE_OPT_FFT_ROWS, FUSE_OPT_FFT_COLS)
        tuned = {k: fuse_get_option(f.ctx, v) for k, v in
                 (("latent_threads", FUSE_OPT_LATENT_THREADS), ("latent_stages", FUSE_OPT_LATENT_STAGES),
                  ("latent_bands", FUSE_OPT_LATENT_BANDS), ("fft_rows", FUSE_OPT_FFT_ROWS),
                  ("fft_cols", FUSE_OPT_FFT_COLS))}
    else:
        tuned = f.autotune(yl, yh, iters=2)        # launch shapes only; results are unchanged

    def step():
        fuse_weights(f.ctx, yh.data_ptr())
        fuse_solve(f.ctx, yl.data_ptr(), yh.data_ptr(), p.iters, 0, None, Z.data_ptr())

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    f.set_option(FUSE_OPT_PROFILE, 1)
    f.profile(FUSE_K_LATENT, reset=True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    lat_ms, lat_n = f.profile(FUSE_K_LATENT)
    _, launches = f.profile(FUSE_K_ALL)
    f.set_option(FUSE_OPT_PROFILE, 0)
    ms = max_over_ranks(ms, dist)
    units = p.H * p.W / 1e6 * p.L_s * p.iters * a.steps * world
    value = job_value(units / world, world, ms / 1e3)

    # end to end through the host-buffer entry point (pinned inputs, Z read back each step)
    e2e = None
    if not a.no_e2e:
        from paper_2210_04184_gb300.fuse import fuse_run_host
        nd = np.float64 if td == torch.float64 else np.float32
        hyl = torch.from_numpy(np.ascontiguousarray(p.Yl, dtype=nd)).pin_memory()
        hyh = torch.from_numpy(np.ascontiguousarray(p.Yh, dtype=nd)).pin_memory()
        hz = torch.empty((p.L_l, p.H, p.W), dtype=td).pin_memory()
        f.set_option(FUSE_OPT_PROFILE, 0)
        for _ in range(max(1, a.warmup)):
            fuse_run_host(f.ctx, hyl.data_ptr(), hyh.data_ptr(), None, p.iters, None, hz.data_ptr())
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            fuse_run_host(f.ctx, hyl.data_ptr(), hyh.data_ptr(), None, p.iters, None, hz.data_ptr())
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dist)
        e2e = {"value": units / dt, "unit": UNIT,
               "h2d_bytes_per_step": hyl.numel() * hyl.element_size() + hyh.numel() * hyh.element_size(),
               "d2h_bytes_per_step": hz.numel() * hz.element_size()}

    fp64 = None
    Z64 = None
    if not a.no_fp64 and meta["dtype"] == "f32":
        fp64, Z64 = fp64_compare(p, meta, f, yl, yh, Z)
    fixed = None
    if not a.no_fixed and rank == 0 and meta["dtype"] == "f32" and p.W % 8 == 0:
        fixed = fixed_point_bench(a, p, meta, yl, yh, Z64)
    sbx = None
    if not a.no_sb and rank == 0 and p.d > 1 and "mask" not in meta:
        sbx = sb_bench(a, p, meta, yl, yh, f)
    grad = None
    if not a.no_grad and rank == 0 and a.workload == "hsms_256":
        grad = grad_bench(a, rank)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    per_launch_ms = lat_ms / max(lat_n, 1)
    traffic = None
    if a.workload.startswith("hsms") and meta["wdtype"] == "bf16" and "hsms" in LATENT_TRAFFIC_PER_PIXEL:
        traffic = LATENT_TRAFFIC_PER_PIXEL["hsms"] * p.H * p.W
    lb = latent_bytes(p, esz, wsz, ssz=2 if a.fixed_state else None)
    if a.fixed_state:
        traffic = None
    achieved = lb / (per_launch_ms / 1e3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": meta["dtype"], "data": "synthetic",
        "config": dict(_config(p, meta, a.workload, world), launch_shapes=tuned),
        "iters_per_s": p.iters * a.steps * world / (ms / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "kernel": "latent_tma_kernel",
                     "algorithmic_bytes_per_launch": lb, "avg_launch_ms": per_launch_ms,
                     "launches": lat_n, "peak_source": peak_src, "nominal_peak": NOMINAL_HBM_GBS},
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "fp64_compare": fp64,
        "conditioning": dict(zip(("A_x_update", "EEt_plus_rho", "F_inverse"), fuse_conditioning(f.ctx))),
        "fixed_point_state": fixed,
        "sb_x_update": sbx,
        "grad": grad,
    }
    if not a.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(p)
    print(json.dumps(out), flush=True)
    f.close()
    if dist:
        dist.destroy_process_group()


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(a.gpus if a.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
    elif a.grad_only:
        import torch
        torch.cuda.set_device(local_rank)
        from paper_2210_04184_gb300 import build as _build
        _build.build()
        out = grad_bench(a, rank)
        if rank == 0:
            print(json.dumps(out), flush=True)
    elif a.workload == "batch64":
        run_batch(a, rank, world, local_rank)
    else:
        run_ours(a, rank, world, local_rank)


if __name__ == "__main__":
    main()
