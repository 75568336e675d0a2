"""Autotuner for the kernel shapes.

Force kernel: for each active-list length bucket (powers of two of the
active fraction), every compiled variant of the context's precision is
timed on a random active subset with CUDA events; the fastest per bucket
forms a table installed with ``nb_set_force_table``.

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


def _time_ms(fn, reps=2):
    import torch

    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_force(s: "_lib.NBody", fractions=(1.0, 1 / 8, 1 / 64, 1 / 1024), seed=7, reps=2,
               use_cache=True):
    """Time every compatible variant for active lists of n * fraction
    particles; install and return the table [(min_active, variant), ...]."""
    import torch

    n = s.n
    prec = s.cfg.precision
    mask = 1 if s.cfg.eps == 0.0 else 0
    key = f"force|{_gpu_key()}|p{prec}|m{mask}|n{n}|" + ",".join(f"{f:g}" for f in fractions)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        table = [tuple(t) for t in cache[key]["table"]]
        s.set_force_table(table)
        return table, cache[key]["timings"]
    dev = torch.device("cuda", torch.cuda.current_device())
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
        best = None
        for v in cands:
            s.set_force_variant(v, 0)
            s.force_jerk_dev(idx, na, acc, jrk)  # warm-up
            ms = _time_ms(lambda: s.force_jerk_dev(idx, na, acc, jrk), reps)
            timings[f"{na}:{v}"] = ms
            if best is None or ms < best[1]:
                best = (v, ms)
        table.append((na, best[0]))
    s.set_force_variant(-1, 0)
    # a bucket applies from its own length upwards until the next larger one
    table.sort(key=lambda t: -t[0])
    table[-1] = (1, table[-1][1])
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
            ms = _time_ms(lambda: b.run(steps), 1)
            timings[f"{v}:{S}"] = ms
            if best is None or ms < best[2]:
                best = (v, S, ms)
    b.set_tuning(best[0], best[1], 0, True)
    if use_cache:
        cache[key] = {"best": [best[0], best[1]], "timings": timings}
        _save_cache(cache)
    return (best[0], best[1]), timings
