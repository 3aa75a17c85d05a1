"""The DRAM traffic that bench.py attaches to its roofline rows comes from a
committed ncu record keyed to the SHA-256 of each kernel's source file and
the headers it inlines: a changed kernel reports no traffic rather than a
stale figure, and a capture of a smaller case is scaled by the units the
launch processes."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def test_source_hash_of_a_file_list_is_the_hash_of_their_concatenation():
    files = ["paper_2111_05778_gb300/csrc/k_mlp_bf16.cu", "paper_2111_05778_gb300/csrc/tc_ptx.cuh"]
    assert bench._src_hash(files) == _hash(files)
    assert bench._src_hash(files[0]) == _hash(files[:1])
    assert bench._src_hash(files) != bench._src_hash(files[0])


def test_traffic_record_lists_existing_sources():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    assert rec["kernels"]
    for name, k in rec["kernels"].items():
        srcs = [k["source"]] if isinstance(k["source"], str) else k["source"]
        for s in srcs:
            assert os.path.exists(os.path.join(ROOT, s)), (name, s)
        assert k["dram_bytes"] > 0 and k["units"] > 0, name


def test_changed_source_gives_no_traffic_and_small_captures_scale(tmp_path, monkeypatch):
    src = "paper_2111_05778_gb300/csrc/k_pipeline.cu"
    good = bench._src_hash([src])
    rec = {"kernels": {
        "k_ok": {"source": [src], "sha256_16": good, "dram_bytes": 1000.0, "units": 10, "full_size": True},
        "k_small": {"source": [src], "sha256_16": good, "dram_bytes": 1000.0, "units": 10, "full_size": False},
        "k_stale": {"source": [src], "sha256_16": "0" * 16, "dram_bytes": 1000.0, "units": 10, "full_size": True},
    }}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    # the record is read from ROOT/profiles; sources are hashed from the real tree
    real_hash = bench._src_hash
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_src_hash", real_hash)
    os.makedirs(os.path.join(str(tmp_path), os.path.dirname(src)), exist_ok=True)
    with open(os.path.join(ROOT, src), "rb") as f, open(os.path.join(str(tmp_path), src), "wb") as g:
        g.write(f.read())
    assert bench.ncu_traffic("k_ok", 123) == 1000.0      # full-size capture: as recorded
    assert bench.ncu_traffic("k_small", 40) == 4000.0    # 100 B per unit x 40 units
    assert bench.ncu_traffic("k_stale", 10) is None      # the kernel changed since the capture
    assert bench.ncu_traffic("k_missing", 10) is None
