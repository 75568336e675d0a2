"""Autotuner for the kernel shapes.

Force kernel: for each active-list length bucket (powers of two of the
active fraction), every compiled variant of the context's precision is
timed on a random active subset with CUDA events (L2 flushed before each
timing), then the fastest few again with smaller persistent grids, which
sets how finely the stream-K split cuts each i-block's j-range (the
j-split); the fastest (variant, grid cap) per bucket forms a table
installed with ``nb_set_force_table``.

Batched kernel: every compatible (variant, steps per launch) pair is timed
on the actual cluster set for a few steps under the CUDA graph; the
fastest is installed with ``nb_batched_set_tuning``.

Results are cached as JSON under ``_build/tune_cache.json`` keyed by the GPU
name, SM count, precision and problem signature, so a second run of the same
workload reuses them.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import _lib, ics

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")


def _gpu_key():
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}"


def _load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


_FLUSH = {}


def _flush_l2():
    """Write 256 MB (more than the 129 MB L2) so that the next timing starts
    from a cold cache, as a force call in a real step does."""
    import torch

    dev = torch.cuda.current_device()
    buf = _FLUSH.get(dev)
    if buf is None:
        buf = _FLUSH[dev] = torch.empty(64 * 1024 * 1024, dtype=torch.float32,
                                        device=torch.device("cuda", dev))
    buf.zero_()


def _time_ms(fn, reps=2, flush=False):
    """Median of reps CUDA-event timings of fn (L2 flushed before each one,
    outside the events, when flush is set)."""
    import torch

    ts = []
    for _ in range(reps):
        if flush:
            _flush_l2()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def grid_caps(num_sms):
    """Caps of the persistent grid searched with each shape: the full grid
    (0), two and one CTA per SM, and half and a quarter of the SMs.  A
    smaller grid gives each CTA a longer contiguous range of (i-block,
    j-tile) units, so fewer i-blocks have their j-range split into stream-K
    segments (less fix-up work) at the cost of fewer busy SMs."""
    return [0, 2 * num_sms, num_sms, num_sms // 2, num_sms // 4]


def tune_force(s: "_lib.NBody", fractions=(1.0, 1 / 8, 1 / 64, 1 / 1024), seed=7, reps=3,
               use_cache=True, finalists=3):
    """For active lists of n * fraction particles, time every compatible
    variant at the full persistent grid, then the `finalists` fastest with
    each cap of grid_caps() (the stream-K j-split), L2 flushed before every
    timing; install and return the table [(min_active, variant, grid_cap),
    ...] and the timings."""
    import torch

    n = s.n
    prec = s.cfg.precision
    mask = _lib.eps_masks(s.cfg.eps)
    key = (f"force2|{_gpu_key()}|p{prec}|m{mask}|n{n}|" +
           ",".join(f"{f:g}" for f in fractions))
    cache = _load_cache() if use_cache else {}
    if key in cache:
        table = [tuple(t) for t in cache[key]["table"]]
        s.set_force_table(table)
        return table, cache[key]["timings"]
    dev = torch.device("cuda", torch.cuda.current_device())
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cands = []
    for v in range(_lib.num_variants()):
        info = _lib.variant_info(v)
        if info["precision"] != prec:
            continue
        try:
            s.set_force_variant(v, 0)
        except _lib.NBodyError:
            continue
        cands.append(v)
    timings = {}
    table = []
    for f in sorted(fractions, reverse=True):
        na = max(1, int(round(n * f)))
        idx = torch.from_numpy(ics.random_active_subset(n, na, seed)).to(dev)
        acc = torch.empty((na, 3), dtype=torch.float64, device=dev)
        jrk = torch.empty_like(acc)

        def run(v, cap):
            s.set_force_variant(v, cap)
            s.force_jerk_dev(idx, na, acc, jrk)  # warm-up (and scratch sizing)
            ms = _time_ms(lambda: s.force_jerk_dev(idx, na, acc, jrk), reps, flush=True)
            timings[f"{na}:{v}:{cap}"] = ms
            return ms

        first = sorted((run(v, 0), v) for v in cands)
        best = (first[0][1], 0, first[0][0])
        for _, v in first[:finalists]:
            for cap in grid_caps(num_sms)[1:]:
                if cap < 1:
                    continue
                ms = run(v, cap)
                if ms < best[2]:
                    best = (v, cap, ms)
        table.append((na, best[0], best[1]))
    s.set_force_variant(-1, 0)
    # a bucket applies from its own length upwards until the next larger one
    table.sort(key=lambda t: -t[0])
    table[-1] = (1,) + tuple(table[-1][1:])
    s.set_force_table(table)
    if use_cache:
        cache[key] = {"table": table, "timings": timings}
        _save_cache(cache)
    return table, timings


def tune_batched(b: "_lib.Batch", steps=50, spl=(1000, 10), use_cache=True):
    """Time every compatible batched variant and steps-per-launch value on
    the batch itself (its state advances by the timed steps); install and
    return the best (variant, steps_per_launch)."""
    sizes = np.diff(b.offsets)
    sig = f"{len(sizes)}:{int(sizes.sum())}:{int((sizes.astype(np.int64) ** 2).sum())}"
    key = f"batched|{_gpu_key()}|p{b.precision}|m{b.mask}|{sig}|steps{steps}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        best = tuple(cache[key]["best"])
        b.set_tuning(best[0], best[1], 0, True)
        return best, cache[key]["timings"]
    timings = {}
    best = None
    for v in range(_lib.num_batched_variants()):
        for S in spl:
            try:
                b.set_tuning(v, S, 0, True)
            except _lib.NBodyError:
                break
            b.run(steps)  # capture + warm-up
            ms = _time_ms(lambda: b.run(steps), 1)  # the ~100 MB state stays in L2
            timings[f"{v}:{S}"] = ms
            if best is None or ms < best[2]:
                best = (v, S, ms)
    b.set_tuning(best[0], best[1], 0, True)
    if use_cache:
        cache[key] = {"best": [best[0], best[1]], "timings": timings}
        _save_cache(cache)
    return (best[0], best[1]), timings
