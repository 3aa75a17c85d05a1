"""The multi-GPU path of bench.py is replicas only (every rank polygonizes
its own mesh; the method needs no exchange): the job's time is the slowest
rank's and its throughput the units of all ranks over that time.  Checked
with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(r, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=r, world_size=world)
    # rank r: 10 steps in 100 (1 + r) ms, 1000 (r + 1) units per step's mesh
    ms, value = bench.aggregate_replicas(100.0 * (1 + r), 1000.0 * (r + 1), 10, world)
    q.put((r, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_summed_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, ms, value in res:
        assert ms == pytest.approx(20.0)               # the slower rank: 200 ms over 10 steps
        assert value == pytest.approx(3000.0 / 0.020)  # 1000 + 2000 units per 20 ms


def test_single_replica_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    ms, value = bench.aggregate_replicas(50.0, 500.0, 5, 1)
    assert ms == pytest.approx(10.0) and value == pytest.approx(50000.0)
