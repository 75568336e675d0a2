"""i-split shards of the Hermite block-step integrator: host logic.

The paper's two-GPU version of its code (Sec. 4, version E) divides the
particles whose forces are computed among the GPUs; every GPU keeps all
particles as sources.  Here each shard is a libnbody context made shard r
of P with nb_shard_set: it owns a contiguous index range, predicts every
particle, evaluates the force and runs the corrector for its slice of the
block's active list, and exports the corrected records of that slice.  The
one exchange of a block step is an all-gather of those records in rank
order, which is the whole active list's records in list order (the list is
ascending and the ranges are contiguous); every shard then imports them.
No counts are exchanged: each shard finds every rank's slice in its own
copy of the active list (nb_shard_offsets).

Two drivers share this module:

* ``ShardGroup``: P shards in one process on one device; each shard
  exports straight into its slice's rows of one buffer, so the all-gather
  is that buffer itself.
* ``RankShard``: one shard per process; the all-gather is
  ``all_gather_records`` over a torch.distributed process group.

Every computation of the method runs in the library's kernels; this module
only partitions, pads and concatenates.
"""
from __future__ import annotations

import numpy as np

from . import _lib

REC = _lib.SHARD_RECORD_DOUBLES


def partition(n: int, nranks: int) -> np.ndarray:
    """Bounds of nranks contiguous, balanced index ranges of n particles:
    rank r owns [b[r], b[r + 1])."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    return np.array([n * r // nranks for r in range(nranks + 1)], dtype=np.int64)


def slice_offsets(act: np.ndarray, bounds: np.ndarray) -> np.ndarray:
    """Offsets of every rank's slice in an ascending active list (what
    nb_shard_offsets computes on the device)."""
    return np.searchsorted(np.asarray(act), np.asarray(bounds), side="left").astype(np.int64)


def all_gather_records(own, counts, group=None):
    """Concatenate the ranks' record rows in rank order over a
    torch.distributed group: rank r contributes `own` (counts[r] rows of
    REC doubles); rows are padded to the largest count for the collective
    and the padding is dropped afterwards."""
    import torch
    import torch.distributed as dist

    counts = [int(c) for c in counts]
    mx = max(counts) if counts else 0
    if mx == 0:
        return own.new_zeros((0, REC))
    pad = own.new_zeros((mx, REC))
    if own.shape[0]:
        pad[: own.shape[0]] = own
    bufs = [torch.empty_like(pad) for _ in counts]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([b[:c] for b, c in zip(bufs, counts)])


class ShardGroup:
    """P shards of one system in one process, on the current CUDA device.

    A block step runs next_block, predict, force of the own slice and
    corrector on every shard, then each exports at its slice's offset of
    one record buffer, and every shard imports the buffer."""

    def __init__(self, m, x, v, nranks: int, **kw):
        import torch

        n = len(m)
        self.n = n
        self.nranks = nranks
        self.bounds = partition(n, nranks)
        self.shards = []
        try:
            for r in range(nranks):
                s = _lib.NBody(m, x, v, **kw)
                self.shards.append(s)
                s.shard_set(nranks, r, self.bounds)
        except Exception:
            self.close()
            raise
        self.rec = torch.empty((n, REC), dtype=torch.float64,
                               device=torch.device("cuda", torch.cuda.current_device()))

    def close(self):
        for s in self.shards:
            s.close()
        self.shards = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self):
        """One block step; returns (t_next, n_active)."""
        blocks = [s.next_block() for s in self.shards]
        t, na = blocks[0]
        if any(b != blocks[0] for b in blocks[1:]):
            raise RuntimeError(f"shards disagree on the block: {blocks}")
        for s in self.shards:
            s.predict(t)
            s.force_jerk_dev(None, na, None, None)
            s.correct(t)
        off = self.shards[0].shard_offsets()
        for r, s in enumerate(self.shards):
            if off[r + 1] > off[r]:
                s.shard_export(self.rec[int(off[r]):])
            else:
                s.shard_export(None)
        for s in self.shards:
            s.shard_import(self.rec, na)
        return t, na

    def get_state(self, want=("x", "v", "a", "jerk", "t_tick", "lev")):
        return self.shards[0].get_state(want=want)

    def counters(self):
        """Interactions evaluated over all shards (each counts its own)."""
        c = [s.counters() for s in self.shards]
        return {"blocks": c[0]["blocks"], "interactions": sum(q["interactions"] for q in c)}


class RankShard:
    """This process's shard of a system split over a torch.distributed
    group (one shard per rank, e.g. one per GPU)."""

    def __init__(self, m, x, v, rank: int, nranks: int, group=None, **kw):
        import torch

        n = len(m)
        self.rank, self.nranks, self.group = rank, nranks, group
        self.bounds = partition(n, nranks)
        self.s = _lib.NBody(m, x, v, **kw)
        self.s.shard_set(nranks, rank, self.bounds)
        own_max = int(self.bounds[rank + 1] - self.bounds[rank])
        self.own = torch.empty((max(own_max, 1), REC), dtype=torch.float64,
                               device=torch.device("cuda", torch.cuda.current_device()))

    def close(self):
        self.s.close()

    def step(self):
        t, na = self.s.next_block()
        self.s.predict(t)
        self.s.force_jerk_dev(None, na, None, None)
        self.s.correct(t)
        off = self.s.shard_offsets()
        cnt = self.s.shard_export(self.own)
        allrec = all_gather_records(self.own[:cnt], np.diff(off), self.group)
        self.s.shard_import(allrec, na)
        return t, na
