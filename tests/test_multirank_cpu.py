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


def _shard_worker(rank, world, port, q):
    """One rank of the i-split exchange on the CPU: the rank finds every
    rank's slice of the block's ascending active list from the partition,
    fills its own slice's records, and the records of all ranks are
    gathered in rank order (the exchange step of the split)."""
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_0909_0879_gb300 import shard

        n = 1000
        bounds = shard.partition(n, world)
        rng = np.random.default_rng(5)  # the same block on every rank
        results = []
        for act in (np.sort(rng.choice(n, 137, replace=False)),  # spread over both ranges
                    np.array([1, 2, 3]),                           # all in rank 0's range
                    np.array([], dtype=np.int64)):                 # empty block
            off = shard.slice_offsets(act, bounds)
            mine = act[off[rank]:off[rank + 1]]
            own = torch.tensor([[i + 0.25 * c for c in range(shard.REC)] for i in mine],
                               dtype=torch.float64).reshape(-1, shard.REC)
            allrec = shard.all_gather_records(own, np.diff(off))
            want = np.array([[i + 0.25 * c for c in range(shard.REC)] for i in act],
                            dtype=np.float64).reshape(-1, shard.REC)
            # import: every active particle's row lands at its index
            state = np.full((n, shard.REC), -1.0)
            state[act] = allrec.numpy()
            results.append((bool(np.array_equal(allrec.numpy(), want)), list(np.diff(off)),
                            float(state.sum())))
        q.put((rank, list(bounds), results))
    finally:
        dist.destroy_process_group()


def test_two_rank_shard_exchange():
    import torch.multiprocessing as mp

    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == out[1][1] == [0, 500, 1000]
    for k in range(3):
        (ok0, c0, s0), (ok1, c1, s1) = out[0][2][k], out[1][2][k]
        assert ok0 and ok1, k
        assert c0 == c1 and sum(c0) == (137, 3, 0)[k]
        assert s0 == s1  # both ranks hold the same state after the import
    assert out[0][2][1][1] == [3, 0]


def test_partition_and_slices():
    from paper_0909_0879_gb300 import shard

    for n, p in ((10, 3), (1, 1), (7, 7), (1 << 20, 8)):
        b = shard.partition(n, p)
        assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
        assert np.diff(b).max() - np.diff(b).min() <= 1
    act = np.array([0, 3, 4, 5, 9])
    assert list(shard.slice_offsets(act, [0, 4, 8, 10])) == [0, 2, 4, 5]
