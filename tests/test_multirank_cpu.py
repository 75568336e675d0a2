"""Host-side logic of the multi-GPU path, run as world_size-2 gloo ranks on
the CPU: independent replicas, whole-job throughput = units of all ranks /
slowest rank's time, and the per-rank seeds give independent clusters."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_0909_0879_gb300 import ics, metrics

        # rank r is slower and does more work; the job rate is total / slowest
        rate, tmax, units = metrics.aggregate_throughput(1.0 + rank, 100.0 * (rank + 1))
        m, x, v = ics.king(2000, 7.0, 1003 + rank)
        q.put((rank, rate, tmax, units, float(x[:10].sum())))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_replica_seeds():
    import torch.multiprocessing as mp

    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, rate, tmax, units, _ in out:
        assert tmax == 2.0 and units == 300.0 and rate == 150.0
    assert out[0][4] != out[1][4]  # the two replicas integrate different clusters


def test_single_process_aggregation_is_local():
    from paper_0909_0879_gb300 import metrics

    assert metrics.aggregate_throughput(2.0, 10.0) == (5.0, 2.0, 10.0)
