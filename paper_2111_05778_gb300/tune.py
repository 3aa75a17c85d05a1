"""Autotuner for batched polygonization: picks the analytic hopper's CTA size
(ray tile: 128, 256 or 512 rays per CTA) and the BF16 engine's GEMM tile (128
or 256 rows per weight K-block) by timing the actual batch, and caches the
choice per GPU and batch signature in a JSON file
($GH_TUNE_CACHE, default ~/.cache/gridhop-gb300/tune.json)."""
from __future__ import annotations

import json
import os

CANDIDATES = [(rb, mt) for rb in (128, 256, 512) for mt in (1, 2)]


def _cache_path():
    return os.environ.get("GH_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gridhop-gb300",
                                                        "tune.json"))


def signature(sdbs, Ns, precision):
    """Batch signature: the multiset of (kind, width, N bucket)."""
    items = []
    for s, n in zip(sdbs, Ns):
        kind = "mlp%d" % s.width if hasattr(s, "width") else "csg"
        bucket = 1 << max(0, (int(n) - 1).bit_length())
        items.append("%s@%d" % (kind, bucket))
    return precision + ":" + ",".join(sorted(items))


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def tune_batch(sdbs, Ns, precision="fp32", eps=None, repeats=2, use_cache=True):
    """Returns (ray_block, mlp_tiles, timings_ms) for this batch."""
    import torch

    from . import gh

    dev = torch.cuda.get_device_name()
    key = dev + "|" + signature(sdbs, Ns, precision)
    cache = _load() if use_cache else {}
    if key in cache:
        c = cache[key]
        return c["ray_block"], c["mlp_tiles"], c.get("timings_ms", {})
    has_mlp = any(hasattr(s, "width") for s in sdbs)
    has_csg = any(not hasattr(s, "width") for s in sdbs)
    cands = [(rb, mt) for rb, mt in CANDIDATES if (has_csg or rb == 256) and
             ((has_mlp and precision == "bf16") or mt == 2)]
    base = gh.polygonize_batch(sdbs, Ns, precision=precision, eps=eps)
    caps = [int(c * 1.05) + 4096 for c in base.counts()]
    timings = {}
    for rb, mt in cands:
        bt = gh.Batch(sdbs, Ns, caps, precision=precision, eps=eps, ray_block=rb, mlp_tiles=mt)
        bt.run(sync=True)
        best = float("inf")
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            bt.run(sync=False)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        timings["%d/%d" % (rb, mt)] = best
    rb, mt = min(cands, key=lambda c: timings["%d/%d" % c])
    cache[key] = {"ray_block": rb, "mlp_tiles": mt, "timings_ms": timings}
    if use_cache:
        _store(cache)
    return rb, mt, timings
