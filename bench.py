"""Benchmark of the grid-hopping polygonizer on one GB300 (or N replicas).

Workload: the neural SDB f(p) = (|p| - 0.6 + 0.1 g(p)) / 1.1, g a seeded
spectrally normalised ReLU MLP 3 -> 256 x 6 -> 1, polygonized on an N = 1024
grid over [-1, 1]^3 (synthetic stand-in for the paper's learned SDBs,
Sec. 5.2).  One step = one whole polygonization (ray hopping, vertex lists,
vertex evaluation, FP32 refinement, Marching Cubes) through gh_polygonize.

Metric: surface cells per second (sign-change cells / ms per mesh), the
headline path being BF16 tensor-core hopping with FP32 refinement; the plain
FP32 path is timed beside it.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (hopper + Marching Cubes) on a
bounded random sample of the same grid's columns on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "neural SDB seed 1 (MLP 3->256x6->1, spectral-normalised, ReLU), N=1024, [-1,1]^3",
    "sdb": "mlp", "seed": 1, "width": 256, "N": 1024,
}
FLOP_PER_EVAL = 2 * (3 * 256 + 5 * 256 * 256 + 256)  # weights only: 657,408


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--N", type=int, default=None, help="grid size (default 1024; smaller for profiling)")
    ap.add_argument("--workload", default="neural", choices=["neural", "batch", "csg", "adjoint", "crossover"],
                    help="neural: one N=1024 neural SDB (default); batch: the 64-item batch, graph-replayed; "
                         "csg: the analytic scene at N=512; adjoint: gh_backward on the N=256 neural mesh")
    args = ap.parse_args()
    if args.N:
        WORKLOAD["N"] = int(args.N)
        WORKLOAD["workload"] = WORKLOAD["workload"].replace("N=1024", "N=%d" % args.N)
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_replicas(total_ms, units, steps, world, device="cpu"):
    """Whole-job throughput of `world` independent replicas (weak scaling:
    each rank polygonizes its own mesh): the slowest rank's time (max over
    ranks of the timed region) and the units of all ranks.  Returns
    (ms per step, units per second).  Needs an initialised process group when
    world > 1 (NCCL on GPUs, gloo in the CPU tests)."""
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([float(total_ms), float(units)], dtype=torch.float64, device=device)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        tot = t.clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        total_ms, units = float(mx[0].item()), float(tot[1].item())
    ms = total_ms / steps
    return ms, units / (ms / 1e3)


# ---------------------------------------------------------------------------
# oracle on the host cores (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(seconds: float, seed: int = 123):
    """Times the FP64 oracle (serial hopper + Marching Cubes) on random columns
    of the workload grid; returns (surface cells per second, cores, sample)."""
    import oracle
    from paper_2111_05778_gb300 import synth

    N, W = WORKLOAD["N"], WORKLOAD["width"]
    o = oracle.mlp(W, synth.MLP_NMID, synth.mlp_params(WORKLOAD["seed"], W).astype(np.float64))
    rng = np.random.default_rng(seed)
    cols_all = rng.permutation(N * N)
    n = 256
    t0 = time.perf_counter()
    _, mr = oracle.polygonize(o, N, cols=cols_all[:n])
    dt = time.perf_counter() - t0
    if dt < seconds:
        n = int(min(len(cols_all), max(n, n * seconds / max(dt, 1e-3))))
        t0 = time.perf_counter()
        _, mr = oracle.polygonize(o, N, cols=cols_all[:n])
        dt = time.perf_counter() - t0
    surf = int(((mr.cases > 0) & (mr.cases < 255)).sum())
    return surf / dt, oracle.num_threads(), "%d uniformly random columns of the N=%d grid (%.1f s, %d surface cells)" % (
        n, N, dt, surf), dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each step is a bounded sample so that --steps K --warmup W ends in minutes
    per_step = max(2.0, min(args.cpu_seconds, 120.0 / max(1, args.steps)))
    for k in range(args.warmup):
        oracle_sample(1.0, seed=900 + k)
    vals, secs = [], []
    for k in range(args.steps):
        v, cores, sample, dt = oracle_sample(per_step, seed=123 + k)
        vals.append(v)
        secs.append(dt)
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": "surface cells/s", "value": value, "unit": "cells/s", "n_gpus": world,
        "steps": len(vals), "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": dict(WORKLOAD),
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def run_ours(args):
    import torch

    from paper_2111_05778_gb300 import gh, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    N, W = WORKLOAD["N"], WORKLOAD["width"]
    params = synth.mlp_params(WORKLOAD["seed"], W)
    sdb = gh.MlpSdb(params, W)
    precision = args.precision
    if precision == "auto":
        precision = "bf16" if _bf16_available(sdb) else "fp32"
    eps = None
    if precision == "bf16":
        eps = sdb.calibrate(N)

    # size the buffers with one synchronous call
    probe = gh.polygonize(sdb, N, precision=precision, eps=eps)
    cap = int(probe.n_tris * 1.05) + 4096
    bufs = gh.Buffers(cap)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step():
        return gh.polygonize_into(sdb, N, bufs, precision=precision, eps=eps, sync=False, stream=stream)

    gh.set_profiling(True)
    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    hop_ms, phases_sum = [], {}
    launches = 0
    for i in range(args.steps):
        ev[i][0].record(stream)
        rc = step()
        ev[i][1].record(stream)
        n_l, ph = gh.last_profile()  # waits for this step's phase events
        launches += n_l
        hop_ms.append(ph.get("hop", float("nan")))
        for k, v in ph.items():
            phases_sum[k] = phases_sum.get(k, 0.0) + v
        flush.zero_()
        assert rc == gh.GH_OK
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    st = bufs.stats_dict()
    assert st["status"] == 0, st
    cells = st["surface_cells"]
    ms, value = aggregate_replicas(total_ms, cells, args.steps, world, device=dev)

    # rooflines of the kernels that dominate the step, from the phase events
    peaks, peak_kind = measured_peaks()
    phase_ms = {k: v / args.steps for k, v in phases_sum.items()}
    kern = kernel_rooflines(precision, st, phase_ms, peaks, peak_kind)
    roof = dict(max(kern, key=lambda r: r["kernel_ms"]))
    roof["note"] = "dominant kernel of the step; all kernels in 'kernels'"

    # end to end through the public API with host buffers
    e2e = e2e_measure(gh, torch, params, W, N, precision, eps, cap, max(2, min(args.steps, 5)), stream)

    line = {
        "metric": "surface cells/s", "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if precision == "bf16" else "f32", "data": "synthetic",
        "config": dict(WORKLOAD, precision="bf16+fp32-refine" if precision == "bf16" else "fp32",
                       l2="256 MB buffer written between timed steps (L2 flush)", replicas=world),
        "ms_per_mesh": ms, "surface_cells": cells, "triangles": st["triangles"], "hop_evals": st["hop_evals"],
        "marked_cells": st["marked_cells"], "unique_vertices": st["unique_vertices"],
        "refined_vertices": st["refined_vertices"],
        "hop_row_utilization": st["hop_evals"] / st["row_slots"] if st.get("row_slots") else None,
        "phases_ms": phase_ms,
        "roofline": roof, "kernels": kern, "clocks": clk, "gpu_launches": launches, "e2e": e2e,
    }
    if precision == "bf16":
        line["fp32_path"] = fp32_companion(gh, torch, sdb, N, bufs, stream, flush)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        v, cores, sample, _ = oracle_sample(args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _src_hash(rel):
    import hashlib

    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(kernel, units):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary (profiles/ncu_traffic.json); scaled by the units the launch
    processes when the capture was a smaller case; None when missing or when
    the kernel's source changed after the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)["kernels"][kernel]
    except (OSError, KeyError, ValueError):
        return None
    if _src_hash(rec["source"]) != rec["sha256_16"]:
        return None
    if rec.get("full_size"):
        return float(rec["dram_bytes"])
    return float(rec["dram_bytes"]) / rec["units"] * units


def kernel_rooflines(precision, st, phase_ms, peaks, peak_kind):
    """One roofline row per compute kernel: achieved = algorithmic FLOPs (f
    evaluations x 2(3W + 5W^2 + W)) / the kernel's event-timed duration."""
    bf16_peak = float(peaks.get("bf16_tflops", 1931.4))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    rows = []

    def row(name, phase, units, bound):
        ms = phase_ms.get(phase)
        if not ms or units <= 0:
            return
        fl = units * FLOP_PER_EVAL
        ach = fl / (ms / 1e3) / 1e12
        peak = bf16_peak if bound == "tensor" else fp32_peak
        rows.append({"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach / peak, "traffic": ncu_traffic(name, units), "kernel_ms": ms,
                     "flop_per_launch": fl, "units_per_launch": units,
                     "peak_source": ("bf16_tflops (%s)" % peak_kind) if bound == "tensor" else
                     "FP32 FFMA: 152 SMs x 128 lanes x 2 FLOP x %.0f MHz (derived)" % sm_max})

    if precision == "bf16":
        row("k_mlp_bf16<256,0,2>", "hop", st["hop_evals"], "tensor")
        row("k_mlp_bf16<256,1,2>", "vertices", st["unique_vertices"], "tensor")
        row("k_pts_mlp_fp32<256,1>", "refine", st["refined_vertices"], "alu")
    else:
        row("k_hop_mlp_fp32<256>", "hop", st["hop_evals"], "alu")
        row("k_pts_mlp_fp32<256,0>", "vertices", st["unique_vertices"], "alu")
    return rows


def _bf16_available(sdb):
    from paper_2111_05778_gb300 import gh

    try:
        sdb.calibrate(64, n_points=4096)
        return True
    except gh.GhError:
        return False


def fp32_companion(gh, torch, sdb, N, bufs, stream, flush, steps=3):
    gh.polygonize_into(sdb, N, bufs, precision="fp32", sync=True, stream=stream)
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gh.polygonize_into(sdb, N, bufs, precision="fp32", sync=False, stream=stream)
        b.record(stream)
        _, ph = gh.last_profile()
        flush.zero_()
        torch.cuda.synchronize()
        ts.append((a.elapsed_time(b), ph.get("hop", float("nan"))))
    st = bufs.stats_dict()
    ms = float(np.mean([t[0] for t in ts]))
    hop = float(np.mean([t[1] for t in ts]))
    return {"ms_per_mesh": ms, "value": st["surface_cells"] / (ms / 1e3), "unit": "cells/s",
            "hop_ms": hop, "hop_tflops": st["hop_evals"] * FLOP_PER_EVAL / (hop / 1e3) / 1e12}


def e2e_measure(gh, torch, params, W, N, precision, eps, cap, steps, stream):
    """Per step: the SDB blob goes host -> device (gh_create_sdb), the mesh is
    polygonized, and the triangle soup comes back into pinned host memory."""
    host_tris = torch.empty((cap, 3, 3), dtype=torch.float32, pin_memory=True)
    bufs = gh.Buffers(cap)
    times, cells, h2d, d2h = [], 0, 0, 0
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sdb = gh.MlpSdb(params, W)
        rc = gh.polygonize_into(sdb, N, bufs, precision=precision, eps=eps, sync=True, stream=stream)
        assert rc == gh.GH_OK
        T = int(bufs.counts[0].item())
        host_tris[:T].copy_(bufs.tri_xyz[:T], non_blocking=True)
        st = bufs.stats.cpu()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sdb.close()
        if i > 0:
            times.append(dt)
        cells = int(st[6])
        h2d = params.nbytes + 32
        d2h = T * 36 + 16 + 128
    ms = float(np.mean(times)) * 1e3
    return {"value": cells / (ms / 1e3), "unit": "cells/s", "ms_per_mesh": ms, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


BATCH_WORKLOAD = {
    "workload": "batch of 64 SDBs (seeds 0..63: even CSG 24 spheres + 8 tori - 4 boxes, odd neural MLP width "
                "64/128/256), N in {128..1024}, one CUDA graph",
}


def run_batch(args):
    """The 64-item batch: hopping in one persistent launch per evaluator
    family, the whole sequence captured in a CUDA graph and replayed."""
    import torch

    from paper_2111_05778_gb300 import gh, synth, tune

    torch.cuda.set_device(0)
    items = synth.batch_items(64)
    sdbs, Ns = [], []
    for kind, seed, N, W in items:
        if kind == "csg":
            s = gh.CsgSdb(synth.csg_prims(seed))
        else:
            s = gh.MlpSdb(synth.mlp_params(seed, W), W)
            s.calibrate(N, n_points=1 << 18)
        sdbs.append(s)
        Ns.append(N)
    precision = "bf16" if args.precision in ("auto", "bf16") else "fp32"
    rb, mt, timings = tune.tune_batch(sdbs, Ns, precision=precision, use_cache=False)
    base = gh.polygonize_batch(sdbs, Ns, precision=precision, ray_block=rb, mlp_tiles=mt)
    caps = [int(c * 1.05) + 4096 for c in base.counts()]
    bt = gh.Batch(sdbs, Ns, caps, precision=precision, ray_block=rb, mlp_tiles=mt)
    bt.capture()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        bt.replay()
        flush.zero_()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    ts = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bt.replay()
        b.record(stream)
        flush.zero_()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    clk = clocks.stop()
    stats = [bt.bufs[i].stats_dict() for i in range(len(sdbs))]
    cells = sum(st["surface_cells"] for st in stats)
    ms = float(np.mean(ts))
    line = {
        "metric": "surface cells/s", "value": cells / (ms / 1e3), "unit": "cells/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if precision == "bf16" else "f32", "data": "synthetic",
        "config": dict(BATCH_WORKLOAD, precision=precision, ray_block=rb, mlp_tiles=mt,
                       l2="256 MB buffer written between timed steps (L2 flush)"),
        "meshes": len(sdbs), "ms_per_mesh": ms / len(sdbs), "surface_cells": cells,
        "triangles": sum(st["triangles"] for st in stats), "autotune_ms": timings, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def _timed(fn, steps, warmup, flush, stream):
    import torch

    for _ in range(warmup):
        fn()
        flush.zero_()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        flush.zero_()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.mean(ts))


def run_csg(args):
    """The analytic scene (CSG seed 0: 24 spheres + 8 tori - 4 boxes) at N = 512, FP32."""
    import torch

    from paper_2111_05778_gb300 import gh, synth

    torch.cuda.set_device(0)
    N = args.N or 512
    sdb = gh.CsgSdb(synth.csg_prims(0))
    probe = gh.polygonize(sdb, N)
    bufs = gh.Buffers(int(probe.n_tris * 1.05) + 4096)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    gh.set_profiling(True)
    phases = {}

    def step():
        gh.polygonize_into(sdb, N, bufs, sync=False, stream=stream)
        _, ph = gh.last_profile()
        for k, v in ph.items():
            phases.setdefault(k, []).append(v)

    clocks = ClockSampler(0)
    ms = _timed(step, args.steps, args.warmup, flush, stream)
    clk = clocks.stop()
    st = bufs.stats_dict()
    line = {"metric": "surface cells/s", "value": st["surface_cells"] / (ms / 1e3), "unit": "cells/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "analytic CSG seed 0 (24 spheres + 8 tori - 4 boxes), N=%d, [-1,1]^3" % N},
            "ms_per_mesh": ms, "phases_ms": {k: float(np.mean(v[args.warmup:] or v)) for k, v in phases.items()},
            "hop_evals": st["hop_evals"], "marked_cells": st["marked_cells"],
            "unique_vertices": st["unique_vertices"], "surface_cells": st["surface_cells"],
            "triangles": st["triangles"], "clocks": clk}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """gh_backward for the C4 workload: the width-256 network of seed 1, its
    N = 256 FP32 mesh, loss = mean over unique vertices of (|v - c| - 0.55)^2."""
    import torch

    from paper_2111_05778_gb300 import gh, synth

    torch.cuda.set_device(0)
    W, N = 256, args.N or 256
    sdb = gh.MlpSdb(synth.mlp_params(1, W), W)
    verts = gh.polygonize(sdb, N, indexed=True).verts  # one vertex per crossing edge, on the device
    c = torch.tensor(np.random.default_rng(4).uniform(-0.05, 0.05, 3), dtype=torch.float32, device="cuda")
    v = verts.clone().requires_grad_(True)
    loss = ((v - c).norm(dim=1) - 0.55).pow(2).mean()
    loss.backward()
    dldv = v.grad.detach()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ms = _timed(lambda: gh.backward(sdb, verts, dldv), args.steps, args.warmup, flush, stream)
    V = verts.shape[0]
    flop = V * 2 * (3 * W + 5 * W * W + W) * 3  # forward, delta chain, weight sums (weights only)
    fp32_peak = 152 * 128 * 2 * 2070e6 / 1e12
    line = {"metric": "adjoint vertices/s", "value": V / (ms / 1e3), "unit": "vertices/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "implicit adjoint, neural SDB seed 1 width 256, N=%d mesh, %d vertices" % (N, V)},
            "roofline": {"bound": "alu", "achieved": flop / (ms / 1e3) / 1e12, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": flop / (ms / 1e3) / 1e12 / fp32_peak, "traffic": None,
                         "kernel": "gh_backward (all kernels)"}}
    print(json.dumps(line), flush=True)


def run_crossover(args):
    """Grid hopping against enumeration (Sec. 2: every lattice point and cell)
    on the same GPU, for the analytic scene, the width-256 network and a
    network of the paper's own architecture (8 layers of width 64, batch
    normalisation folded, lambda = 1.5), over N (the paper's Sec. 5
    comparisons, here with both methods on the GB300)."""
    import torch

    from paper_2111_05778_gb300 import gh, synth

    torch.cuda.set_device(0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    pp, pw, pl, plam, _ = synth.paper_network(0)
    cases = [("csg", gh.CsgSdb(synth.csg_prims(0)), (64, 128, 256, 512, 1024)),
             ("mlp256", gh.MlpSdb(synth.mlp_params(1, 256), 256), (64, 128, 256, 512)),
             ("paper_net_8x64_bn", gh.paper_mlp(pp, pw, pl, plam), (64, 128, 256, 512))]
    for name, sdb, Ns in cases:
        for N in Ns:
            res = {"sdb": name, "N": N}
            variants = [("hop_fp32", "fp32", "hop"), ("enum_fp32", "fp32", "enum")]
            if name != "csg":
                variants.insert(1, ("hop_bf16", "bf16", "hop"))
            for key, prec, meth in variants:
                eps = sdb.calibrate(N, n_points=1 << 18) if prec == "bf16" else None
                probe = gh.polygonize(sdb, N, precision=prec, eps=eps, method=meth)
                bufs = gh.Buffers(int(probe.n_tris * 1.05) + 4096)
                gh.polygonize_into(sdb, N, bufs, precision=prec, eps=eps, method=meth)
                ms = _timed(lambda: gh.polygonize_into(sdb, N, bufs, precision=prec, eps=eps, sync=False,
                                                       stream=stream, method=meth),
                            max(1, args.steps // 2), 1, flush, stream)
                res[key + "_ms"] = ms
                res[key + "_evals"] = bufs.stats_dict()["hop_evals"]
            rows.append(res)
            print(json.dumps(res), flush=True)
    print(json.dumps({"workload": "crossover", "rows": rows}), flush=True)


def main():
    args = parse()
    if args.workload == "crossover":
        run_crossover(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "csg":
        run_csg(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
