"""Benchmark of the grid-hopping polygonizer on one GB300 (or N replicas).

Headline workload: the neural SDB f(p) = (|p| - 0.6 + 0.1 g(p)) / 1.1, g a
seeded spectrally normalised ReLU MLP 3 -> 256 x 6 -> 1, polygonized on an
N = 1024 grid over [-1, 1]^3 (synthetic stand-in for the paper's learned SDBs,
Sec. 5.2).  One step = one whole polygonization (ray hopping, vertex lists,
vertex evaluation, FP32 refinement, Marching Cubes) through gh_polygonize.

Metric: surface cells per second (sign-change cells / ms per mesh), the
headline path being BF16 tensor-core hopping with FP32 refinement; the plain
FP32 path is timed beside it.  After the headline's timed region the other
workloads are timed the same way and reported under "workloads": the sphere
at N = 64, the analytic CSG scene at N = 512, the batch of 64 SDBs replayed
as one CUDA graph, and the implicit adjoint at N = 256.  Last, on the host
cores, the CPU baseline leg times the FP64 oracle on bounded samples of every
workload and compares the GPU results with the oracle's on those samples
("accuracy").  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (hopper + Marching Cubes) on a
bounded random sample of the same grid's columns on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
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


def mlp_flop(width, n_mid=5):
    """Algorithmic FLOP of one neural-SDB evaluation (weights only)."""
    return 2 * (3 * width + n_mid * width * width + width)


FLOP_PER_EVAL = mlp_flop(256)  # 657,408

# FLOP of one primitive's exact distance as written (an FMA counts 2, a
# square root 1), rotation into the local frame included; plus one min/max of
# the fold.  One analytic evaluation = the whole fold over all primitives.
PRIM_FLOP = {0: 11, 1: 29, 2: 38, 3: 30, 4: 32, 5: 45, 6: 50}


def csg_flop(prims):
    return int(sum(PRIM_FLOP[int(t)] for t in np.asarray(prims)[:, 0]))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16", "bf16x6"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true", help="time the headline workload only")
    ap.add_argument("--no-companions", action="store_true",
                    help="skip the other precisions of the headline workload (for profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--N", type=int, default=None, help="grid size (default 1024; smaller for profiling)")
    ap.add_argument("--workload", default="neural", choices=["neural", "batch", "csg", "adjoint", "crossover"],
                    help="neural: one N=1024 neural SDB (default, with the other workloads after it); "
                         "batch / csg / adjoint: that workload alone; crossover: hopping vs enumeration")
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
# The oracle on the host cores: the CPU baseline leg and the reference arm.
# Everything below that runs oracle code is called only from cpu_leg() (after
# every GPU timed region) and from run_reference().
# ---------------------------------------------------------------------------
def _oracle_mlp(seed, width):
    import oracle
    from paper_2111_05778_gb300 import synth

    return oracle.mlp(width, synth.MLP_NMID, synth.mlp_params(seed, width).astype(np.float64))


def oracle_sample(seconds: float, seed: int = 123, osdb=None):
    """Times the FP64 oracle (serial hopper + Marching Cubes) on random columns
    of the headline grid; returns (surface cells per second, cores, sample,
    seconds, columns, MC result)."""
    import oracle

    N, W = WORKLOAD["N"], WORKLOAD["width"]
    o = osdb if osdb is not None else _oracle_mlp(WORKLOAD["seed"], W)
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
    return (surf / dt, oracle.num_threads(),
            "%d uniformly random columns of the N=%d grid (%.1f s, %d surface cells)" % (n, N, dt, surf), dt,
            np.sort(cols_all[:n]), mr)


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
        v, cores, sample, dt, _, _ = oracle_sample(per_step, seed=123 + k)
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


def _parity():
    tests = os.path.join(ROOT, "tests")
    if tests not in sys.path:
        sys.path.insert(0, tests)
    import parity

    return parity


def _acc(st, N, stats=None):
    """The accuracy record of one comparison (parity.compare, reporting form)."""
    out = {"cells_compared": st["cells"], "tie_cells_1e-6h": st["tie_cells"],
           "exact_zero_cells": st["exact_zero_cells"], "fp32_sign_flip_cells": st["sign_flip_cells"],
           "fp32_sign_flip_cells_outside_band": st["sign_flip_outside_band"],
           "mismatched_cells": st["mismatched_cells"],
           "mismatched_triangles": st["mismatched_tris"], "vertices_compared": st["verts"],
           "vertices_over_tolerance": st["vertices_over_tol"], "max_vertex_err_over_h": st["max_err_over_h"],
           "share_within_1e-4h": st["bare_frac"], "delta32": st["delta32"]}
    if stats is not None and N > 1:
        out["hops_per_N2log2N"] = stats["hop_evals"] / (N * N * math.log2(N))
    return out


def _timed_oracle(fn, threads=0):
    import oracle

    oracle.set_threads(threads)
    t0 = time.perf_counter()
    r = fn()
    dt = time.perf_counter() - t0
    oracle.set_threads(0)
    return dt, r


def cpu_leg(ctx, seconds):
    """The oracle on bounded samples of every workload (all host cores, and
    one core for the small ones), and the GPU results compared with the
    oracle's on the same samples.  Returns (cpu_baseline record of the
    headline, accuracy of the headline, {workload: {"oracle": ..,
    "accuracy": ..}})."""
    import oracle

    par = _parity()
    out = {}
    # ---- headline: random columns of the N = 1024 grid ------------------------
    c2 = ctx["c2"]
    N = WORKLOAD["N"]
    o2 = _oracle_mlp(WORKLOAD["seed"], WORKLOAD["width"])
    v, cores, sample, dt, cols, mr = oracle_sample(seconds, osdb=o2)
    hr_cols = oracle.hop(o2, N, cols=cols[:512])
    evals_per_s = float(hr_cols.col_evals.sum()) / _timed_oracle(lambda: oracle.hop(o2, N, cols=cols[:512]))[0]
    cpu = {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample,
           "full_mesh_s_extrapolated": c2["stats"]["surface_cells"] / v,
           "enum_s_extrapolated": 8.0 * N ** 3 / evals_per_s,
           "note": "ghop = the oracle's serial hopper + Marching Cubes; enum = Marching Cubes on all N^3 cells "
                   "(8 evaluations each), extrapolated from the measured evaluation rate"}
    inside = lambda c: np.isin(c // N, cols)
    acc = {}
    for prec, m in c2["meshes"].items():
        st = par.compare(m, o2, N, ref=mr, restrict_cells=inside, gsdb=c2["gsdb"], check=False, gprec=prec)
        acc[prec] = _acc(st, N, m.stats)
    acc["sample"] = "the CPU baseline's %d columns" % cols.size
    # ---- sphere N = 64: the whole grid, all cores and one core ---------------
    if "c0" in ctx:
        c = ctx["c0"]
        o = oracle.csg(c["prims"])
        t_all, (hr, mrr) = _timed_oracle(lambda: oracle.polygonize(o, c["N"]))
        t_one, _ = _timed_oracle(lambda: oracle.polygonize(o, c["N"]), threads=1)
        e_all, er = _timed_oracle(lambda: oracle.enum(o, c["N"]))
        e_one, _ = _timed_oracle(lambda: oracle.enum(o, c["N"]), threads=1)
        st = par.compare(c["mesh"], o, c["N"], ref=mrr, gsdb=c["gsdb"], check=False)
        out["C0"] = {"oracle": {"ghop_s": t_all, "ghop_s_1core": t_one, "enum_s": e_all, "enum_s_1core": e_one,
                                "cores": cores, "hop_evals": int(hr.col_evals.sum())},
                     "accuracy": dict(_acc(st, c["N"], c["mesh"].stats), sample="every cell")}
    # ---- CSG N = 512: sampled columns and one slab, all cores and one core ----
    if "c1" in ctx:
        c = ctx["c1"]
        n1 = c["N"]
        o = oracle.csg(c["prims"])
        rng = np.random.default_rng(5)
        cs = np.sort(rng.choice(n1 * n1, 4000, replace=False))
        t_all, (_, mrr) = _timed_oracle(lambda: oracle.polygonize(o, n1, cols=cs))
        t_one, _ = _timed_oracle(lambda: oracle.polygonize(o, n1, cols=cs[:1000]), threads=1)
        k0 = n1 // 2 + 7
        e_all, er = _timed_oracle(lambda: oracle.enum(o, n1, kmin=k0, kmax=k0 + 1))
        st = par.compare(c["mesh"], o, n1, ref=mrr, restrict_cells=lambda x: np.isin(x // n1, cs), gsdb=c["gsdb"],
                         check=False)
        st2 = par.compare(c["mesh"], o, n1, ref=er, restrict_cells=lambda x: (x % n1) == k0, gsdb=c["gsdb"],
                          check=False)
        out["C1"] = {"oracle": {"ghop_s_extrapolated": t_all * n1 * n1 / cs.size,
                                "ghop_s_1core_extrapolated": t_one * n1 * n1 / 1000,
                                "enum_s_extrapolated": e_all * n1, "cores": cores,
                                "sample": "4000 random columns (1000 on one core); enum: one z-slab"},
                     "accuracy": {"columns": _acc(st, n1, c["mesh"].stats), "slab_k%d" % k0: _acc(st2, n1)}}
    # ---- batch: 16 random columns of every item -------------------------------
    if "c3" in ctx:
        t_sum, worst, rows = 0.0, {}, 0
        for kind, seed, n, w, gsdb, m, prims in ctx["c3"]["items"]:
            o = oracle.csg(prims) if kind == "csg" else _oracle_mlp(seed, w)
            rng = np.random.default_rng(1000 + seed)
            cs = np.sort(rng.choice(n * n, 16, replace=False))
            dt_i, (_, mrr) = _timed_oracle(lambda: oracle.polygonize(o, n, cols=cs))
            t_sum += dt_i * n * n / cs.size
            st = par.compare(m, o, n, ref=mrr, restrict_cells=lambda x: np.isin(x // n, cs), gsdb=gsdb,
                             check=False)
            rows += st["cells"]
            for key in ("mismatched_cells", "mismatched_triangles", "vertices_over_tolerance",
                        "max_vertex_err_over_h"):
                a = _acc(st, n)[key]
                worst[key] = max(worst.get(key, 0), a)
        worst["cells_compared"] = rows
        out["C3"] = {"oracle": {"ghop_s_extrapolated": t_sum, "cores": cores,
                                "sample": "16 random columns of each of the 64 items"},
                     "accuracy": dict(worst, sample="16 random columns of each item (worst item shown)")}
    # ---- adjoint: the FP64 adjoint on the same vertices ---------------------------
    if "c4" in ctx:
        c = ctx["c4"]
        V = c["verts"].cpu().numpy().astype(np.float64)
        G = c["dldv"].cpu().numpy().astype(np.float64)
        t_all, g64 = _timed_oracle(lambda: oracle.np_adjoint(c["params"].astype(np.float64), c["W"], 5, V, G))
        g = c["grad"].cpu().numpy().astype(np.float64)
        scale = np.abs(g64).max()
        rel = np.abs(g - g64) / np.maximum(np.abs(g64), 1e-2 * scale)
        out["C4"] = {"oracle": {"adjoint_s": t_all, "cores": cores, "kind": "numpy FP64 adjoint (oracle.np_adjoint)"},
                     "accuracy": {"max_rel_err": float(rel.max()), "median_rel_err": float(np.median(rel)),
                                  "metric": "|g - g64| / max(|g64|, 1e-2 max|g64|) over all parameters"}}
    return cpu, acc, out
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




def _events(stream):
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _timed(fn, steps, warmup, flush, stream):
    """Mean CUDA-event ms of fn over `steps` runs after `warmup` runs, the L2
    flushed (a 256 MB buffer written) between runs."""
    import torch

    for _ in range(warmup):
        fn()
        flush.zero_()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        a, b = _events(stream)
        a.record(stream)
        fn()
        b.record(stream)
        flush.zero_()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.mean(ts))


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
        precision = "bf16x6" if _bf16_available(sdb) else "fp32"
    eps = None
    if precision in ("bf16", "bf16x6"):
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
    ev = [_events(stream) for _ in range(args.steps)]
    phases_sum = {}
    launches = 0
    for i in range(args.steps):
        ev[i][0].record(stream)
        rc = step()
        ev[i][1].record(stream)
        n_l, ph = gh.last_profile()  # waits for this step's phase events
        launches += n_l
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
    if precision != "fp32":
        e2e["eps"] = "calibrated once per SDB before the timed region (gh_sdb_calibrate), not in this number"
        cal = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sdb.calibrate(N)
            cal.append((time.perf_counter() - t0) * 1e3)
        e2e["calibrate_ms"] = float(np.median(cal))
        e2e["value_with_calibration"] = cells / ((e2e["ms_per_mesh"] + e2e["calibrate_ms"]) / 1e3)

    line = {
        "metric": "surface cells/s", "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "bf16", "data": "synthetic",
        "config": dict(WORKLOAD, precision={"bf16": "bf16+fp32-refine", "bf16x6": "bf16+split-bf16x6-refine",
                                            "fp32": "fp32"}[precision],
                       l2="256 MB buffer written between timed steps (L2 flush)", replicas=world),
        "ms_per_mesh": ms, "surface_cells": cells, "triangles": st["triangles"], "hop_evals": st["hop_evals"],
        "hops_per_N2log2N": st["hop_evals"] / (N * N * math.log2(N)),
        "marked_cells": st["marked_cells"], "unique_vertices": st["unique_vertices"],
        "refined_vertices": st["refined_vertices"],
        "hop_row_utilization": st["hop_evals"] / st["row_slots"] if st.get("row_slots") else None,
        "phases_ms": phase_ms,
        "roofline": roof, "kernels": kern, "clocks": clk, "gpu_launches": launches, "e2e": e2e,
    }
    ctx = {}
    if precision != "fp32" and not args.no_companions:
        line["fp32_path"] = companion(gh, torch, sdb, N, bufs, stream, flush, "fp32")
        other = "bf16" if precision == "bf16x6" else "bf16x6"
        line["bf16_fp32_refine_path" if other == "bf16" else "bf16x6_refine_path"] = companion(
            gh, torch, sdb, N, bufs, stream, flush, other, eps)
    solo = rank == 0 and world == 1
    if solo and not args.no_cpu_baseline:
        meshes = {precision: gh.polygonize(sdb, N, precision=precision, eps=eps, keys=True, cells=True)}
        for extra in ("fp32", "bf16", "bf16x6"):
            if precision != "fp32" and extra not in meshes:
                meshes[extra] = gh.polygonize(sdb, N, precision=extra, eps=None if extra == "fp32" else eps,
                                              keys=True, cells=True)
        ctx["c2"] = {"gsdb": sdb, "meshes": meshes, "stats": st}
    if solo and not args.no_workloads:
        line["workloads"] = {}
        for name, fn in (("C0", work_c0), ("C1", work_c1), ("C3", work_c3), ("C4", work_c4)):
            rec, c = fn(args, flush, stream)
            line["workloads"][name] = rec
            ctx[name.lower()] = c
    if solo and not args.no_cpu_baseline:
        cpu, acc, per = cpu_leg(ctx, args.cpu_seconds)
        line["cpu_baseline"] = cpu
        line["accuracy"] = acc
        for name, rec in per.items():
            line["workloads"].setdefault(name, {}).update(rec)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _src_hash(rel):
    """First 16 hex digits of the SHA-256 of a source file, or of the
    concatenation of a list of them (a kernel's file and the headers it
    inlines)."""
    import hashlib

    h = hashlib.sha256()
    for r in [rel] if isinstance(rel, str) else rel:
        with open(os.path.join(ROOT, r), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


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

    if precision in ("bf16", "bf16x6"):
        row("k_mlp_bf16<256,0,2>", "hop", st["hop_evals"], "tensor")
        row("k_mlp_bf16<256,1,2>", "vertices", st["unique_vertices"], "tensor")
        if precision == "bf16":
            row("k_pts_mlp_fp32<256,1>", "refine", st["refined_vertices"], "alu")
        elif phase_ms.get("refine"):
            # six BF16 tensor products per hidden-layer product (executed FLOP)
            fl = st["refined_vertices"] * 6 * 2 * 5 * 256 * 256
            ms = phase_ms["refine"]
            ach = fl / (ms / 1e3) / 1e12
            rows.append({"kernel": "k_mlp_x6<256,0>", "bound": "tensor", "achieved": ach, "peak": bf16_peak,
                         "unit": "TFLOP/s", "frac": ach / bf16_peak, "traffic": ncu_traffic("k_mlp_x6<256,0>",
                         st["refined_vertices"]), "kernel_ms": ms, "flop_per_launch": fl,
                         "units_per_launch": st["refined_vertices"],
                         "peak_source": "bf16_tflops (%s)" % peak_kind})
    else:
        row("k_hop_mlp_fp32<256>", "hop", st["hop_evals"], "alu")
        row("k_pts_mlp_fp32<256,0>", "vertices", st["unique_vertices"], "alu")
    mc = mesh_write_row(st, WORKLOAD["N"], phase_ms.get("mc"), peaks, peak_kind)
    if mc:
        rows.append(mc)
    return rows


def _bf16_available(sdb):
    from paper_2111_05778_gb300 import gh

    try:
        sdb.calibrate(64, n_points=4096)
        return True
    except gh.GhError:
        return False


def companion(gh, torch, sdb, N, bufs, stream, flush, precision="fp32", eps=None, steps=3):
    """The same workload in another precision, a few steps (not the headline)."""
    gh.polygonize_into(sdb, N, bufs, precision=precision, eps=eps, sync=True, stream=stream)
    ts, phs = [], []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gh.polygonize_into(sdb, N, bufs, precision=precision, eps=eps, sync=False, stream=stream)
        b.record(stream)
        _, ph = gh.last_profile()
        flush.zero_()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
        phs.append(ph)
    st = bufs.stats_dict()
    assert st["status"] == 0, st
    ms = float(np.mean(ts))
    ph = {k: float(np.mean([p[k] for p in phs])) for k in phs[0]}
    out = {"precision": precision, "ms_per_mesh": ms, "value": st["surface_cells"] / (ms / 1e3), "unit": "cells/s",
           "phases_ms": ph, "hop_tflops": st["hop_evals"] * FLOP_PER_EVAL / (ph["hop"] / 1e3) / 1e12}
    if precision == "bf16x6":
        peaks, peak_kind = measured_peaks()
        W = WORKLOAD["width"]
        tensor = st["refined_vertices"] * 6 * 2 * 5 * W * W  # six BF16 products per hidden-layer product
        ach = tensor / (ph["refine"] / 1e3) / 1e12
        bf = float(peaks.get("bf16_tflops", 1917.8))
        out["refine_roofline"] = {
            "kernel": "k_mlp_x6<256,0>", "bound": "tensor", "achieved": ach, "peak": bf, "unit": "TFLOP/s",
            "frac": ach / bf, "traffic": None, "kernel_ms": ph["refine"], "units_per_launch": st["refined_vertices"],
            "flop_per_launch": tensor, "peak_source": "bf16_tflops (%s)" % peak_kind,
            "fp32_equivalent_tflops": st["refined_vertices"] * FLOP_PER_EVAL / (ph["refine"] / 1e3) / 1e12}
    return out


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




# ---------------------------------------------------------------------------
# The other workloads, each timed on its own after the headline's timed region
# ---------------------------------------------------------------------------
def _alu_row(kernel, flop, ms, peaks):
    fp32_peak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    ach = flop / (ms / 1e3) / 1e12
    return {"kernel": kernel, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": ach / fp32_peak, "traffic": None, "kernel_ms": ms, "flop_per_launch": flop,
            "peak_source": "FP32: 152 SMs x 128 lanes x 2 FLOP x max SM clock (derived)"}


def mesh_write_row(st, N, ms, peaks, peak_kind):
    """k_mc (Marching Cubes on the marked cells) against HBM: algorithmic
    bytes = the soup written (36 B per triangle) + the marks read (8 B per
    marked cell) + the vertex list read once (8 B key + 4 B value per lattice
    vertex) + the line offsets (4 B per lattice line)."""
    if not ms:
        return None
    T, M, V = st["triangles"], st["marked_cells"], st["unique_vertices"]
    byts = 36 * T + 8 * M + 12 * V + 4 * (N + 1) ** 2
    ach = byts / (ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    return {"kernel": "k_mc", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": ncu_traffic("k_mc", M), "kernel_ms": ms, "bytes_per_launch": byts,
            "mesh_bytes": 36 * T, "peak_source": "hbm_gbs (%s)" % peak_kind}


def _csg_workload(prims, N, args, flush, stream, name):
    from paper_2111_05778_gb300 import gh

    sdb = gh.CsgSdb(prims)
    probe = gh.polygonize(sdb, N)
    bufs = gh.Buffers(int(probe.n_tris * 1.05) + 4096)
    gh.set_profiling(True)
    phases = {}

    def step():
        gh.polygonize_into(sdb, N, bufs, sync=False, stream=stream)
        _, ph = gh.last_profile()
        for k, v in ph.items():
            phases.setdefault(k, []).append(v)

    clocks = ClockSampler(0)
    steps = max(args.steps, 10)
    ms = _timed(step, steps, args.warmup, flush, stream)
    clk = clocks.stop()
    st = bufs.stats_dict()
    assert st["status"] == 0, st
    ph = {k: float(np.mean(v[-steps:])) for k, v in phases.items()}
    peaks, peak_kind = measured_peaks()
    kern = [_alu_row("k_hop_csg", st["hop_evals"] * csg_flop(prims), ph["hop"], peaks),
            _alu_row("k_eval_vertices_csg", st["unique_vertices"] * csg_flop(prims), ph["vertices"], peaks),
            mesh_write_row(st, N, ph["mc"], peaks, peak_kind)]
    rec = {"workload": name, "ms_per_mesh": ms, "value": st["surface_cells"] / (ms / 1e3), "unit": "cells/s",
           "dtype": "f32", "steps": steps, "phases_ms": ph, "hop_evals": st["hop_evals"],
           "hops_per_N2log2N": st["hop_evals"] / (N * N * math.log2(N)), "marked_cells": st["marked_cells"],
           "unique_vertices": st["unique_vertices"], "surface_cells": st["surface_cells"],
           "triangles": st["triangles"], "flop_per_eval": csg_flop(prims),
           "roofline": dict(max(kern, key=lambda r: r["kernel_ms"])), "kernels": kern, "clocks": clk}
    mesh = gh.polygonize(sdb, N, keys=True, cells=True)
    return rec, {"prims": prims, "gsdb": sdb, "mesh": mesh, "N": N}


def work_c0(args, flush, stream):
    from paper_2111_05778_gb300 import synth

    return _csg_workload(synth.sphere_prims(0.5), 64, args, flush, stream,
                         "analytic sphere |p| - 0.5, N=64, [-1,1]^3, FP32")


def work_c1(args, flush, stream):
    from paper_2111_05778_gb300 import synth

    return _csg_workload(synth.csg_prims(0), args.N if args.workload == "csg" and args.N else 512, args, flush,
                         stream, "analytic CSG seed 0 (24 spheres + 8 tori - 4 boxes), N=512, [-1,1]^3, FP32")


BATCH_WORKLOAD = ("batch of 64 SDBs (seeds 0..63: even CSG 24 spheres + 8 tori - 4 boxes, odd neural MLP width "
                  "64/128/256), N in {128..1024}, one CUDA graph")


def work_c3(args, flush, stream):
    """The 64-item batch: hopping in one persistent launch per evaluator
    family, the whole sequence captured in a CUDA graph and replayed."""
    from paper_2111_05778_gb300 import gh, synth, tune

    items = synth.batch_items(64)
    sdbs, Ns, prims_of = [], [], []
    t0 = time.perf_counter()
    for kind, seed, N, W in items:
        if kind == "csg":
            p = synth.csg_prims(seed)
            s = gh.CsgSdb(p)
        else:
            p = None
            s = gh.MlpSdb(synth.mlp_params(seed, W), W)
            s.calibrate(N, n_points=1 << 18)
        sdbs.append(s)
        Ns.append(N)
        prims_of.append(p)
    setup_s = time.perf_counter() - t0
    precision = "bf16x6" if args.precision == "auto" else args.precision
    rb, mt, timings = tune.tune_batch(sdbs, Ns, precision=precision, use_cache=False)
    base = gh.polygonize_batch(sdbs, Ns, precision=precision, ray_block=rb, mlp_tiles=mt)
    caps = [int(c * 1.05) + 4096 for c in base.counts()]
    bt = gh.Batch(sdbs, Ns, caps, precision=precision, ray_block=rb, mlp_tiles=mt)
    bt.capture()
    clocks = ClockSampler(0)
    steps = max(args.steps, 5)
    ms = _timed(bt.replay, steps, args.warmup, flush, stream)
    clk = clocks.stop()
    stats = [bt.bufs[i].stats_dict() for i in range(len(sdbs))]
    assert all(st["status"] == 0 for st in stats)
    cells = sum(st["surface_cells"] for st in stats)
    peaks, peak_kind = measured_peaks()
    tensor_flop = sum((st["hop_evals"] + st["unique_vertices"]) * mlp_flop(W)
                      for (kind, _, _, W), st in zip(items, stats) if kind == "mlp") if precision != "fp32" else 0
    refine_flop = sum(st["refined_vertices"] * mlp_flop(W) for (kind, _, _, W), st in zip(items, stats)
                      if kind == "mlp")
    if precision == "bf16x6":
        tensor_flop += 6 * refine_flop  # six BF16 products per split-BF16 evaluation
        note = ("BF16 tensor FLOP executed by the neural items (hop and vertex evaluations, and six BF16 products "
                "per split-BF16 refinement) over the whole batch time (analytic items, lists and Marching Cubes "
                "included in the time)")
    else:
        note = ("BF16 tensor FLOP of the neural items (hop + vertex evaluations) over the whole batch time "
                "(analytic items, FP32 refinement (%.2f TFLOP), lists and Marching Cubes included in the time)"
                % (refine_flop / 1e12))
    bf16_peak = float(peaks.get("bf16_tflops", 1917.8))
    ach = tensor_flop / (ms / 1e3) / 1e12
    rec = {"workload": BATCH_WORKLOAD, "ms_per_batch": ms, "ms_per_mesh": ms / len(sdbs),
           "value": cells / (ms / 1e3), "unit": "cells/s", "dtype": "f32" if precision == "fp32" else "bf16",
           "steps": steps, "meshes": len(sdbs), "surface_cells": cells,
           "triangles": sum(st["triangles"] for st in stats), "ray_block": rb, "mlp_tiles": mt,
           "autotune_ms": timings, "setup_s": setup_s,
           "roofline": {"kernel": "whole batch (graph replay)", "bound": "tensor", "achieved": ach, "peak": bf16_peak,
                        "unit": "TFLOP/s", "frac": ach / bf16_peak, "traffic": None, "note": note,
                        "peak_source": "bf16_tflops (%s)" % peak_kind},
           "clocks": clk}
    chk = gh.polygonize_batch(sdbs, Ns, precision=precision, keys=True, cells=True, ray_block=rb, mlp_tiles=mt)
    ctx = {"items": [(kind, seed, N, W, sdbs[b], chk.mesh(b), prims_of[b])
                     for b, (kind, seed, N, W) in enumerate(items)]}
    bt.close()
    return rec, ctx


def work_c4(args, flush, stream):
    """gh_backward for the C4 workload: the width-256 network of seed 1, its
    N = 256 FP32 mesh, loss = mean over unique vertices of (|v - c| - 0.55)^2."""
    import torch

    from paper_2111_05778_gb300 import gh, synth

    W, N = 256, 256
    params = synth.mlp_params(1, W)
    sdb = gh.MlpSdb(params, W)
    verts = gh.polygonize(sdb, N, indexed=True).verts  # one vertex per crossing edge, on the device
    c = torch.tensor(np.random.default_rng(4).uniform(-0.05, 0.05, 3), dtype=torch.float32, device="cuda")
    v = verts.clone().requires_grad_(True)
    loss = ((v - c).norm(dim=1) - 0.55).pow(2).mean()
    loss.backward()
    dldv = v.grad.detach()
    clocks = ClockSampler(0)
    steps = max(args.steps, 10)
    ms = _timed(lambda: gh.backward(sdb, verts, dldv), steps, args.warmup, flush, stream)
    clk = clocks.stop()
    V = verts.shape[0]
    flop = V * mlp_flop(W) * 3  # forward, delta chain, weight sums (weights only)
    peaks, _ = measured_peaks()
    row = _alu_row("gh_backward (all kernels)", flop, ms, peaks)
    rec = {"workload": "implicit adjoint, neural SDB seed 1 width 256, N=%d mesh, %d vertices" % (N, V),
           "metric": "adjoint vertices/s", "ms": ms, "value": V / (ms / 1e3), "unit": "vertices/s", "dtype": "f32",
           "steps": steps, "vertices": V, "roofline": row, "clocks": clk}
    grad = gh.backward(sdb, verts, dldv)
    torch.cuda.synchronize()
    return rec, {"verts": verts, "dldv": dldv, "grad": grad, "params": params, "W": W}
def run_crossover(args):
    """Grid hopping against enumeration (Sec. 2: every lattice point and cell)
    and, for the analytic scene, continuation (Sec. 2: the surface crawled
    from seed points, here one left of every primitive's centre) on the same
    GPU, for the analytic scene, the width-256 network and a network of the
    paper's own architecture (8 layers of width 64, batch normalisation
    folded, lambda = 1.5), over N (the paper's Sec. 5 comparisons, here with
    every method on the GB300)."""
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
            if name == "csg":
                seeds = synth.csg_prims(0)[:, 2:5].copy()
                seeds[:, 0] -= 0.3
                probe = gh.polygonize_cont(sdb, N, seeds)
                bufs = gh.Buffers(int(probe.n_tris * 1.05) + 4096)
                gh.polygonize_cont_into(sdb, N, seeds, bufs)
                res["cont_fp32_ms"] = _timed(lambda: gh.polygonize_cont_into(sdb, N, seeds, bufs, sync=False,
                                                                             stream=stream),
                                             max(1, args.steps // 2), 1, flush, stream)
                res["cont_fp32_evals"] = bufs.stats_dict()["hop_evals"]
                res["cont_surface_cells"] = bufs.stats_dict()["surface_cells"]
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


def run_single(args):
    """One of the other workloads alone, as its own bench line."""
    import torch

    torch.cuda.set_device(0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    fn = {"csg": work_c1, "batch": work_c3, "adjoint": work_c4}[args.workload]
    rec, _ = fn(args, flush, stream)
    ms = rec.get("ms_per_mesh", rec.get("ms_per_batch", rec.get("ms")))
    if args.workload == "batch":
        ms = rec["ms_per_batch"]
    line = {"metric": rec.get("metric", "surface cells/s"), "value": rec["value"], "unit": rec["unit"],
            "n_gpus": 1, "steps": rec["steps"], "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"],
            "data": "synthetic", "config": {"workload": rec["workload"],
                                            "l2": "256 MB buffer written between timed steps (L2 flush)"},
            "roofline": rec["roofline"], "clocks": rec["clocks"], "detail": rec}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "crossover":
        run_crossover(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("batch", "csg", "adjoint"):
        run_single(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
