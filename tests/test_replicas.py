"""The N > 1 path of bench.py (independent replicas) with world_size 2 on CPU (gloo).

The solver does not shard; N ranks run the same workload with their own seeds. What the ranks
share is host-side: the barrier around the timed region, the maximum of the timings over ranks
and the whole-job throughput. Each rank here reports a different timing; both must see the
maximum and the same aggregated throughput.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.replica_barrier(world)
        ms = 10.0 + 5.0 * rank            # rank 1 is slower
        ms_max = bench.replica_max(ms, world, "cpu")
        value = bench.replica_throughput(1000, world, ms_max, steps=5)
        bench.replica_barrier(world)
        out[rank] = (ms_max, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_agree_on_the_slowest_rank():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    ms_max, value = out[0]
    assert ms_max == 15.0
    assert value == pytest.approx(1000 * 2 / (15.0 / 5 / 1e3))


def test_single_rank_is_identity():
    import bench
    assert bench.replica_max(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(100, 1, 2.0, 2) == pytest.approx(100 / 1e-3)
