"""Multi-GPU is replicas only: each rank runs the whole workload and the bench reports the
nodes of all ranks over the slowest rank's time.  The host logic of that aggregation runs
here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [1.5, 2.5][rank]                      # rank 1 is the slow replica
        t = bench.reduce_max(ms, dist, "cpu")
        out[rank] = (t, bench.replica_rate(world, 1000, t * 1e-3))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_nodes():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, rate = out[r]
        assert t == 2.5                            # both ranks agree on the max
        assert rate == pytest.approx(2 * 1000 / 2.5e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.0) == 3.0
    assert bench.replica_rate(1, 163842, 0.00066) == pytest.approx(248.245, rel=1e-4)
