#!/usr/bin/env python3
"""Throughput benchmark: G pair-interactions/s of the direct-summation
force + jerk hot path at N = 1,048,576.

Workload: a King W0 = 7 cluster (seeded, equal masses, Henon units),
eps = 1e-4, advanced by 4th-order Hermite steps with a shared step
dt = 2^-10 so that every particle is active in every step.  One timed step
is one pass of the whole path: block scheduling, predictor (split
precision on the FP32 pipe from the FP64 state, writing the j-records),
force + jerk of all N active particles against all N, corrector (FP64
position and velocity update).  An interaction is one (i, j) pair
evaluation; a step evaluates N^2 of them.

Output: one JSON line (rank 0).  `value` is whole-job interactions/s from
CUDA events on the library's stream with inputs resident in HBM; `e2e` is
the same through the C ABI with host buffers (state uploaded and downloaded
every step; from the initial state, after the same warm-up steps, so that
it times the same steps of the integration); `roofline` puts the force
kernel's FP32 arithmetic against the FP32 peak; `cpu_baseline` times the
FP64 oracle on the host cores on a bounded sample.  With `--impl reference` the oracle alone is timed.

Multi-GPU (torchrun): every rank integrates its own independent cluster
(seed 1003 + rank); no collective is on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0909_0879_gb300 import ics, metrics  # noqa: E402

N_DEFAULT = 1 << 20
EPS = 1e-4
W0 = 7.0
LEV_SHARED = 10
METRIC = "G pair-interactions/s (acc+jerk, N=1M)"
UNIT = "Ginteractions/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=6)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="ds", choices=["ds", "fp32"])
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--no-energy", action="store_true", help="skip the FP64 energy check")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--e2e-steps", type=int, default=0,
                   help="steps of the end-to-end leg (0 = as many as --steps)")
    p.add_argument("--variant", type=int, default=-1,
                   help="king1m: force shape; batched: batched shape (skips the tuner)")
    p.add_argument("--grid", type=int, default=0)
    p.add_argument("--batched-steps", type=int, default=1000,
                   help="batched: shared steps per timed run")
    p.add_argument("--workload", default="king1m",
                   choices=["king1m", "shared1024", "block65536", "batched", "adjoint",
                            "nsweep", "symplectic", "isplit"],
                   help="king1m is the headline; the others time the remaining workloads "
                        "and print their own JSON line")
    p.add_argument("--block-steps", type=int, default=0,
                   help="block65536: stop after this many block steps (0 = run to t = 1/8)")
    p.add_argument("--precisions", default="ds,fp32",
                   help="workloads other than king1m: comma-separated precisions to run")
    p.add_argument("--shards", type=int, default=2,
                   help="isplit: shards of the i-split run on this GPU")
    p.add_argument("--sweep", action="store_true",
                   help="also time single evaluations at active fractions 2^-10..1")
    p.add_argument("--relayout-every", type=int, default=0,
                   help="king1m: re-store the particles in a fresh spatial order every K "
                        "block steps (nb_set_relayout_every; 0 = keep the initial order)")
    p.add_argument("--oracle-replay", action="store_true",
                   help="block65536: the FP64 oracle replays the GPU's schedule to t = 1/8 "
                        "and compares |dE/E| (minutes of CPU work)")
    return p.parse_args()


def workload_name(n):
    return f"king_w0_7_n{n}_eps1e-4_hermite_shared_dt2^-{LEV_SHARED}_all_active"


# ------------------------------------------------------------------ clocks

REASON_BITS = {
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
    0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
    0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
    0x100: "display_clock_setting",
}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.gpu),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [q.strip() for q in ln.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[3], 16) if parts[3].startswith("0x") else int(parts[3])
            except ValueError:
                continue
            for b, name in REASON_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- roofline


def force_traffic_from_profile(n):
    """DRAM bytes per force launch from the committed ncu record
    (profiles/force_jerk_ds_traffic.json), if it was taken on the current
    force-kernel source at this N; otherwise None."""
    path = os.path.join(ROOT, "profiles", "force_jerk_ds_traffic.json")
    src = os.path.join(ROOT, "paper_0909_0879_gb300", "csrc", "nb_force.cu")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if rec.get("source_sha256") != cur or int(rec.get("n", -1)) != n:
        return None
    return float(rec["dram_bytes_per_launch"])


def peak_info(num_sms):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    src = "fallback max SM clock 2070 MHz"
    if os.path.exists(path):
        try:
            mp = json.load(open(path))
            if mp.get("sm_max_mhz"):
                sm_max = float(mp["sm_max_mhz"])
                src = "sm_max_mhz from MEASURED_PEAKS.json"
        except Exception:
            pass
    return metrics.fp32_peak_tflops(num_sms, sm_max), sm_max, src


# ------------------------------------------------------------- CPU leg


def cpu_baseline(m, x, v, n, seconds, keep=False):
    """Time the FP64 oracle's force + jerk for a bounded sample of
    i-particles against all n j-particles on every host core.  With keep,
    the sample's indices and the oracle's acceleration and jerk come back
    too (keys "idx", "acc", "jerk")."""
    from oracle import oracle as O

    O.build()
    cores = O.max_threads()
    rng = np.random.default_rng(7)
    probe = np.sort(rng.choice(n, 32, replace=False))
    t0 = time.perf_counter()
    O.force_jerk(m, x, v, EPS, idx=probe)
    dt = time.perf_counter() - t0
    rate = 32 * n / max(dt, 1e-6)
    ns = int(min(n, max(64, rate * seconds / n)))
    ns = max(cores, ns - ns % cores)
    sample = np.sort(rng.choice(n, ns, replace=False))
    t0 = time.perf_counter()
    ra, rj = O.force_jerk(m, x, v, EPS, idx=sample)
    dt = time.perf_counter() - t0
    out = {"value": ns * n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{ns} random i-particles x {n} j-particles, FP64 acc+jerk, "
                     f"{dt:.1f} s on {cores} OpenMP threads",
           "seconds": dt}
    if keep:
        out.update(idx=sample, acc=ra, jerk=rj)
    return out


def force_error(acc, jerk, ra, rj, cond=None):
    """Errors of GPU force + jerk rows against the FP64 oracle's on the same
    particles: per-particle e_i = |da_i| / max(|a_i|, 1e-3 rms|a|) (max and
    99th percentile), norm-wise ||da|| / ||a||, and, with cond = (sum_j
    |f_ij|, sum_j |jerk_ij|) on the first rows, the condition-relative
    |da_i| / sum_j |f_ij|."""
    def per(g, r):
        sc = np.sqrt(np.mean(np.sum(r * r, 1)))
        return np.linalg.norm(g - r, axis=1) / np.maximum(np.linalg.norm(r, axis=1), 1e-3 * sc)

    ea, ej = per(acc, ra), per(jerk, rj)
    out = {"acc_max_ei": float(ea.max()), "acc_p99_ei": float(np.quantile(ea, 0.99)),
           "jerk_max_ei": float(ej.max()), "jerk_p99_ei": float(np.quantile(ej, 0.99)),
           "acc_norm": float(np.linalg.norm(acc - ra) / np.linalg.norm(ra)),
           "jerk_norm": float(np.linalg.norm(jerk - rj) / np.linalg.norm(rj))}
    if cond is not None:
        k = len(cond[0])
        out["acc_cond_max"] = float((np.linalg.norm(acc[:k] - ra[:k], axis=1) / cond[0]).max())
        out["jerk_cond_max"] = float((np.linalg.norm(jerk[:k] - rj[:k], axis=1) / cond[1]).max())
    return out


def _oracle_beside(work, units, unit, sample):
    """The FP64 oracle timed beside a GPU workload: `work` runs a bounded
    sample of the workload's own work in the oracle on every host core;
    `units` of it, reported per second in `unit`."""
    from oracle import oracle as O

    O.build()
    t0 = time.perf_counter()
    work()
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": unit, "cores": O.max_threads(), "kind": "oracle",
            "sample": sample, "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n = args.n
    m, x, v = ics.king(n, W0, 1003)
    steps = []
    cb = None
    per = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(m, x, v, n, per)
        if s >= args.warmup:
            steps.append(r)
        cb = r
    vals = [r["value"] for r in steps]
    val = float(np.mean(vals))
    tot_s = sum(r["seconds"] for r in steps)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot_s / len(steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(n), "n": n, "eps": EPS,
                      "note": "FP64 CPU oracle; each step a bounded i-sample of one "
                              "force+jerk evaluation against all N"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                            "sample": cb["sample"]},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------- GPU leg


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_0909_0879_gb300 import _lib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n
    m, x, v = ics.king(n, W0, 1003 + rank)
    # store the particles in the library's spatial layout (balanced bisection
    # leaves of 256, one per force-kernel tile); the system is unchanged
    perm = _lib.spatial_order(x, 256)
    m, x, v = m[perm], x[perm], v[perm]
    stream = torch.cuda.current_stream(dev)
    s = _lib.NBody(m, x, v, eps=EPS, precision=args.precision, block_steps=False,
                   lev_shared=LEV_SHARED, stream=stream)
    if args.variant >= 0 or args.grid > 0:
        s.set_force_variant(args.variant, args.grid)
    if args.relayout_every > 0:
        s.set_relayout_every(args.relayout_every)
    props = torch.cuda.get_device_properties(dev)
    num_sms = props.multi_processor_count
    st0 = s.get_state()  # the initial state, for the force-error check

    E0 = None
    if not args.no_energy:
        E0 = s.energy()[2]
    # L2 flush buffer: larger than the 129 MB L2
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step(record):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        flush.zero_()
        ev[0].record(stream)
        t, na = s.next_block()
        s.predict(t)
        ev[1].record(stream)
        s.force_jerk_dev(None, na, None, None)
        ev[2].record(stream)
        s.correct(t)
        ev[3].record(stream)
        return ev, na

    for _ in range(args.warmup):
        one_step(False)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    l0 = s.launch_count()
    r0 = s.storage_order()[1]
    evs = []
    inter = 0
    for _ in range(args.steps):
        ev, na = one_step(True)
        evs.append(ev)
        inter += na * n
    torch.cuda.synchronize(dev)
    launches = s.launch_count() - l0
    relayouts = s.storage_order()[1] - r0
    clocks = sampler.stop() if sampler else None
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    force_ms = [e[1].elapsed_time(e[2]) for e in evs]
    rate, t_total, inter_all = metrics.aggregate_throughput(sum(step_ms) / 1e3, inter, dev)
    value = rate / 1e9

    dE = None
    if E0 is not None:
        E1 = s.energy()[2]
        dE = abs(E1 - E0) / abs(E0)

    # end to end through the C ABI with host buffers in pinned memory:
    # upload the state, step, download the state, every step.  The leg
    # starts again from the initial state and takes the same warm-up steps
    # untimed, so that it times the same stretch of the integration as the
    # device leg: the particles are stored in the spatial order of their
    # initial positions, and as they move the far field's tile boxes grow
    # and each step takes a little longer.
    pinned = {}
    for k, a in st0.items():
        t = torch.empty(a.shape, dtype=getattr(torch, a.dtype.name), pin_memory=True)
        pinned[k] = t.numpy()
        pinned[k][...] = a
    st = pinned
    e2e_steps = args.e2e_steps if args.e2e_steps > 0 else max(1, args.steps)
    h2d = sum(a.nbytes for a in st.values())
    d2h = h2d
    for _ in range(args.warmup):
        s.set_state(st)
        s.step()
        s.get_state(out=st)
    torch.cuda.synchronize(dev)
    # the clocks of this leg too: after the timed steps a long run can
    # meet the power limit here
    e2e_sampler = ClockSampler(local_rank) if rank == 0 else None
    if e2e_sampler:
        e2e_sampler.start()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(st)
        s.step()
        s.get_state(out=st)
    torch.cuda.synchronize(dev)
    e2e_t = time.perf_counter() - t0
    e2e_clocks = e2e_sampler.stop() if e2e_sampler else None
    e2e_val = e2e_steps * n * n / e2e_t / 1e9
    if world > 1:
        e2e_val = metrics.aggregate_throughput(e2e_t, e2e_steps * n * n, dev)[0] / 1e9

    sweep = None
    if args.sweep:
        sweep = []
        for k in range(10, -1, -1):
            na = max(1, n >> k)
            idx = torch.from_numpy(ics.random_active_subset(n, na, 3000 + k)).to(dev)
            acc = torch.empty((na, 3), dtype=torch.float64, device=dev)
            jrk = torch.empty_like(acc)
            s.force_jerk_dev(idx, na, acc, jrk)
            ts = []
            for _ in range(3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.force_jerk_dev(idx, na, acc, jrk)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(e0.elapsed_time(e1))
            ms = float(np.median(ts))
            sweep.append({"active_fraction": f"2^-{k}", "n_act": na, "ms": ms,
                          "ginter_s": na * n / ms / 1e6})

    if rank != 0:
        s.close()
        return 0

    # Force error against the FP64 oracle, outside the timed region: the
    # initial state, all N particles evaluated in the bench's launch
    # configuration (identity i-list of length N, the same built-in shape
    # and grid as the timed force call), compared on the oracle's sample.
    s.set_state(st0)
    s.predict(0.0)
    d_idx = torch.arange(n, dtype=torch.int32, device=dev)
    d_acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
    d_jrk = torch.empty_like(d_acc)
    s.force_jerk_dev(d_idx, n, d_acc, d_jrk)
    torch.cuda.synchronize(dev)
    force_s = float(np.mean(force_ms)) / 1e3
    achieved = metrics.FLOPS_PER_INTERACTION * n * n / force_s / 1e12
    peak, sm_max, peak_src = peak_info(num_sms)
    traffic = force_traffic_from_profile(n) if args.precision == "ds" else None
    clk_mhz = clocks.get("sm_mhz") if clocks else None
    cpu = None
    ferr = None
    if not args.no_cpu:
        from oracle import oracle as O

        cpu = cpu_baseline(m, x, v, n, args.cpu_seconds, keep=True)
        samp = cpu.pop("idx")
        ra, rj = cpu.pop("acc"), cpu.pop("jerk")
        cpu.pop("seconds", None)
        sel = torch.from_numpy(samp).to(dev)
        ga = d_acc[sel].cpu().numpy()
        gj = d_jrk[sel].cpu().numpy()
        kc = min(1024, len(samp))
        cond = O.force_jerk_abs(m, x, v, EPS, idx=samp[:kc])
        ferr = force_error(ga, gj, ra, rj, cond)
        ferr["sample"] = (f"the CPU baseline's {len(samp)} random particles (condition sums on "
                          f"the first {kc}), initial state; GPU: all N evaluated as in a timed "
                          f"step")
        if sweep is not None:
            # each active fraction of the sweep at the initial state: the same
            # random subsets, 256 of their particles against the oracle
            for row, k in zip(sweep, range(10, -1, -1)):
                na = row["n_act"]
                sub = ics.random_active_subset(n, na, 3000 + k)
                d_sub = torch.from_numpy(sub).to(dev)
                sa = torch.empty((na, 3), dtype=torch.float64, device=dev)
                sj = torch.empty_like(sa)
                s.force_jerk_dev(d_sub, na, sa, sj)
                torch.cuda.synchronize(dev)
                pick = np.sort(np.random.default_rng(4000 + k).choice(na, min(na, 256),
                                                                       replace=False))
                ra_k, rj_k = O.force_jerk(m, x, v, EPS, idx=sub[pick])
                e = force_error(sa.cpu().numpy()[pick], sj.cpu().numpy()[pick], ra_k, rj_k)
                row["force_err"] = {q: e[q] for q in ("acc_max_ei", "acc_norm", "jerk_max_ei")}
    del d_acc, d_jrk, d_idx
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32-ds" if args.precision == "ds" else "f32",
        "data": "synthetic",
        "config": {
            "workload": workload_name(n), "n": n, "eps": EPS, "W0": W0,
            "integrator": "hermite4 shared dt, all active", "precision": args.precision,
            "parallelism": f"replicas x{world} (independent clusters per GPU)",
            "l2": "flushed between timed steps (256 MB write outside the events)",
            "seed": "1003 + rank",
            "layout": "particles stored in nb_spatial_order (balanced bisection, 256 per leaf)"
                      + (f"; re-stored in the order of the current positions every "
                         f"{args.relayout_every} block steps (nb_set_relayout_every)"
                         if args.relayout_every > 0 else ""),
            "relayouts_timed": relayouts,
        },
        "dE_over_E": dE,
        "dE_note": f"FP64 GPU energy before warm-up and after {args.warmup + args.steps} steps "
                   f"of dt 2^-{LEV_SHARED}" if dE is not None else None,
        "roofline": {
            "bound": "alu",
            "achieved": achieved,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": traffic,
            "kernel": "force_jerk_kernel (+ fix-up) per force evaluation, CUDA events on the "
                      "library stream",
            "flops_per_interaction": metrics.FLOPS_PER_INTERACTION,
            "peak_def": f"{num_sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz ({peak_src})",
            "frac_at_measured_clock": (achieved / metrics.fp32_peak_tflops(num_sms, clk_mhz)
                                       if clk_mhz else None),
            "frac_60flop_convention": achieved / metrics.FLOPS_PER_INTERACTION
            * metrics.FLOPS_PER_INTERACTION_CONVENTION / peak,
        },
        "force_ms": float(np.mean(force_ms)),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": int(e2e_steps),
                "clocks": e2e_clocks,
                "note": "nb_set_state + nb_step + nb_get_state with host arrays in pinned "
                        "memory, wall clock; from the initial state after the same warm-up "
                        "steps as the device leg"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "force_err": ferr,
    }
    if sweep is not None:
        out["sweep"] = sweep
    print(json.dumps(out), flush=True)
    s.close()
    return 0


# ------------------------------------------------------- other workloads


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_shared1024(args):
    """N = 1024 equal-mass Plummer (seed 1001), eps = 1e-3, shared dt = 1/256
    for one time unit (256 steps): interactions/s and conservation, FP32 and
    DS."""
    import torch

    from paper_0909_0879_gb300 import _lib

    n, eps, lev, steps = 1024, 1e-3, 8, 256
    m, x, v = ics.plummer(n, 1001)
    out = {"metric": "G pair-interactions/s (acc+jerk, Hermite shared dt, N=1024)",
           "unit": UNIT, "workload": "plummer_n1024_eps1e-3_dt2^-8_t1", "results": {}}
    for prec in args.precisions.split(","):
        with _lib.NBody(m, x, v, eps=eps, precision=prec, block_steps=False, lev_shared=lev) as s:
            E0 = s.energy()[2]
            L0 = (m[:, None] * np.cross(x, v)).sum(0)
            e0, e1 = _events(torch)
            e0.record()
            for _ in range(steps):
                s.step()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st = s.get_state(want=("x", "v"))
            E1 = s.energy()[2]
        P = (m[:, None] * st["v"]).sum(0)
        L = (m[:, None] * np.cross(st["x"], st["v"])).sum(0)
        # the same 256 steps device-resident (CUDA-graph replays of 32 steps,
        # no host synchronisation per step); bit for bit the same states
        with _lib.NBody(m, x, v, eps=eps, precision=prec, block_steps=False, lev_shared=lev) as s:
            e2, e3 = _events(torch)
            e2.record()
            nblk, _ = s.run_blocks(1.0)
            e3.record()
            torch.cuda.synchronize()
            ms_dev = e2.elapsed_time(e3)
            same = bool(np.array_equal(s.get_state(want=("x",))["x"], st["x"]))
        out["results"][prec] = {"value": steps * n * n / ms / 1e6, "ms": ms,
                                "dE_over_E": abs(E1 - E0) / abs(E0),
                                "dP": float(np.abs(P).max()), "dL": float(np.abs(L - L0).max()),
                                "device_resident": {"value": nblk * n * n / ms_dev / 1e6,
                                                    "ms": ms_dev, "steps": nblk,
                                                    "same_state_as_host_loop": same},
                                "note": "value/ms: host-driven nb_step loop (one host "
                                        "synchronisation per step); device_resident: "
                                        "nb_run_blocks"}
    if not args.no_cpu:
        from oracle import oracle as O

        out["cpu_baseline"] = _oracle_beside(
            lambda: O.hermite_shared(m, x, v, eps, lev, steps), steps * n * n / 1e9, UNIT,
            "the FP64 oracle's shared-step Hermite loop, the same 256 steps")
    print(json.dumps(out), flush=True)
    return 0


def block_energy_replay(_lib, m, x, v, eps, t_end_tick):
    """Energy error of the block-step workload against the FP64 oracle in
    replay mode: the GPU (split precision, host-driven steps) records its
    schedule (block time and ordered active list of every block step) to
    t_end, when all particles are synchronised; the oracle starts from the
    same state and levels and takes the same steps.  The energy pass is
    |dE/E|_gpu <= 2 max(|dE/E|_oracle, 1e-10)."""
    from oracle import oracle as O

    kw = dict(eps=eps, precision="ds", eta=0.01, eta_start=0.01, lev_min=3, lev_max=20)
    sched = []
    with _lib.NBody(m, x, v, **kw) as s:
        lev0 = s.get_state(want=("lev",))["lev"].copy()
        E0 = s.energy()[2]
        while True:
            st = s.get_state(want=("t_tick", "lev"))
            due = st["t_tick"] + (1 << (20 - st["lev"].astype(np.int64)))
            if due.min() > t_end_tick:
                break
            t, na = s.next_block()
            act = s.active()
            s.predict(t)
            s.force_jerk_dev(None, na, None, None)
            s.correct(t)
            sched.append((int(round(t * 2**20)), act.astype(np.int64)))
        xg = s.get_state(want=("x",))["x"]
        E1 = s.energy()[2]
    t0 = time.perf_counter()
    orc = O.HermiteState(m, x, v, eps, eta=0.01, eta_start=0.01, lev_min=3, lev_max=20)
    lev_agree = float(np.mean(orc.lev == lev0))
    orc.lev[:] = lev0  # the GPU's initial levels (equal except at thresholds)
    E0o = orc.energy()[2]
    for tn, act in sched:
        orc.step(replay=(tn, act))
    E1o = orc.energy()[2]
    dg, do = abs(E1 - E0) / abs(E0), abs(E1o - E0o) / abs(E0o)
    return {"block_steps": len(sched), "dE_over_E_gpu": dg, "dE_over_E_oracle": do,
            "pass": bool(dg <= 2 * max(do, 1e-10)),
            "max_abs_dx": float(np.abs(xg - orc.x).max()),
            "initial_levels_equal": lev_agree, "oracle_s": time.perf_counter() - t0,
            "oracle_threads": O.max_threads(),
            "note": "GPU split precision, host-driven steps; the oracle (FP64, every "
                    "interaction) replays the GPU's schedule from the same initial levels"}


def block_force_errors(_lib, m, x, v, eps, precs, checkpoints=(0, 5, 15), ns=4096):
    """Force + jerk errors of the block-step workload against the FP64
    oracle: at the given block steps (from the start), the GPU's force on
    ns sampled particles (seed 2002) at the predicted state, against the
    oracle's on the same state (predicted in FP64 by the oracle from the
    GPU's stored state)."""
    from oracle import oracle as O

    n = len(m)
    sample = np.sort(np.random.default_rng(2002).choice(n, ns, replace=False)).astype(np.int32)
    rows = {}
    for prec in precs:
        rows[prec] = []
        with _lib.NBody(m, x, v, eps=eps, precision=prec, eta=0.01, lev_min=3,
                        lev_max=20) as s:
            done = 0
            for k in checkpoints:
                while done < k:
                    s.step()
                    done += 1
                st = s.get_state()
                t, na = s.next_block()
                s.predict(t)
                dt = (int(round(t * 2**20)) - st["t_tick"]) * 2.0**-20
                xp, vp = O.predict(st["x"], st["v"], st["a"], st["jerk"], dt)
                acc, jerk = s.force_jerk(sample)
                ra, rj = O.force_jerk(m, xp, vp, eps, idx=sample)
                cond = O.force_jerk_abs(m, xp, vp, eps, idx=sample)
                r = force_error(acc, jerk, ra, rj, cond)
                r.update(block_step=k, t=t, n_act=na)
                rows[prec].append(r)
                s.force_jerk_dev(None, na, None, None)
                s.correct(t)
                done += 1
    return {"rows": rows,
            "sample": f"{ns} random particles (seed 2002) at the predicted state of block "
                      f"steps {list(checkpoints)}, FP64 oracle on the same state"}


def run_block65536(args):
    """N = 65536 Plummer with Salpeter masses (seed 1002), eps = 1e-4, Aarseth
    block steps (eta = 0.01, levels 3..20) to t = 1/8: interactions/s over
    the run, block-step count, active-list histogram, |dE/E| at t = 1/8
    (all particles synchronised), FP32 and DS."""
    import torch

    from paper_0909_0879_gb300 import _lib

    n, eps = 65536, 1e-4
    m, x, v = ics.plummer(n, 1002, masses=ics.salpeter_masses(n, 1002))
    out = {"metric": "G pair-interactions/s (acc+jerk, Hermite block steps, N=65536)",
           "unit": UNIT, "workload": "plummer_salpeter_n65536_eps1e-4_eta0.01_t0.125",
           "results": {}}
    t_end = 1 << 17
    max_blocks = args.block_steps if args.block_steps > 0 else 1 << 62
    for prec in args.precisions.split(","):
        with _lib.NBody(m, x, v, eps=eps, precision=prec, eta=0.01, lev_min=3, lev_max=20) as s:
            E0 = s.energy()[2]
            dev_res = None
        if True:
            # device-resident block steps (CUDA-graph replays): the fused
            # form and the general scheduler, each from the initial state
            # (at most --block-steps of them when given)
            dev_res = {}
            for mode in ("auto", "general"):
                with _lib.NBody(m, x, v, eps=eps, precision=prec, eta=0.01, lev_min=3,
                                lev_max=20) as s:
                    s.set_block_mode(mode)
                    e0, e1 = _events(torch)
                    c0 = s.counters()
                    l0 = s.launch_count()
                    t0 = time.perf_counter()
                    e0.record()
                    nblk, _ = s.run_blocks(t_end * 2.0**-20, max(0, args.block_steps))
                    e1.record()
                    torch.cuda.synchronize()
                    wall_dev = time.perf_counter() - t0
                    ms_dev = e0.elapsed_time(e1)
                    c1 = s.counters()
                    E_dev = s.energy()[2]
                    dev_res[s.last_block_path()] = {
                        "value": (c1["interactions"] - c0["interactions"]) / ms_dev / 1e6,
                        "ms": ms_dev, "wall_s": wall_dev, "block_steps": nblk,
                        "launches_per_block": (s.launch_count() - l0) / max(1, nblk),
                        "dE_over_E": (abs(E_dev - E0) / abs(E0)) if args.block_steps == 0
                        else None}
        with _lib.NBody(m, x, v, eps=eps, precision=prec, eta=0.01, lev_min=3, lev_max=20) as s:
            hist = {}
            blocks = 0
            t0 = time.perf_counter()
            e0, e1 = _events(torch)
            e0.record()
            tick = 0
            while tick < t_end and blocks < max_blocks:
                t, na = s.step()
                tick = int(round(t * 2**20))
                blocks += 1
                b = int(np.log2(max(1, na)))
                hist[b] = hist.get(b, 0) + 1
            e1.record()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            ms = e0.elapsed_time(e1)
            cnt = s.counters()
            E1 = s.energy()[2] if tick >= t_end else float("nan")
        out["results"][prec] = {
            "value": cnt["interactions"] / ms / 1e6, "ms": ms, "wall_s": wall,
            "block_steps": blocks, "interactions": cnt["interactions"],
            "clamped": cnt["clamped"], "dE_over_E": abs(E1 - E0) / abs(E0),
            "n_act_log2_histogram": {str(k): v for k, v in sorted(hist.items())},
            "device_resident": dev_res,
            "note": "value/ms: host-driven nb_step loop; device_resident: nb_run_blocks"}
    if not args.no_cpu:
        out["force_err"] = block_force_errors(_lib, m, x, v, eps, args.precisions.split(","))
        if args.oracle_replay:
            out["energy_vs_oracle_replay"] = block_energy_replay(_lib, m, x, v, eps, t_end)
        out["cpu_baseline"] = cpu_baseline(m, x, v, n, 3.0)
    print(json.dumps(out), flush=True)
    return 0


def batched_oracle_checks(_lib, O, off, m, x, v, tuned, steps, n_force=64, n_energy=64):
    """The batched form against the FP64 oracle: the per-particle force and
    jerk errors of the batch's first evaluation on n_force sampled
    clusters, and the energy error over `steps` shared steps of 1/256 from
    the initial state on n_energy of them, GPU (tuned shape) beside the
    oracle's Hermite loop on the same clusters."""
    nc = len(off) - 1
    rng = np.random.default_rng(2004)
    fc = np.sort(rng.choice(nc, n_force, replace=False))
    ec = fc[:n_energy]
    out = {}
    for prec, (var, spl) in tuned.items():
        with _lib.Batch(off, m, x, v, eps=1e-3, lev_shared=8, precision=prec) as b:
            st0 = b.get_state()
            k0, w0 = b.energy()
            b.set_tuning(var, min(spl, steps), 0, True)
            b.run(steps)
            k1, w1 = b.energy()
        ea, ej, na, nj = [], [], [], []
        ca = []
        for c in fc:
            sl = slice(off[c], off[c + 1])
            ra, rj = O.force_jerk(m[sl], x[sl], v[sl], 1e-3)
            cond = O.force_jerk_abs(m[sl], x[sl], v[sl], 1e-3)
            e = force_error(st0["a"][sl], st0["jerk"][sl], ra, rj, cond)
            ea.append(e["acc_max_ei"]); ej.append(e["jerk_max_ei"])
            na.append(e["acc_norm"]); nj.append(e["jerk_norm"])
            ca.append(e["acc_cond_max"])
        dE_gpu = np.abs((k1 + w1) - (k0 + w0)) / np.abs(k0 + w0)
        dE_orc = []
        for c in ec:
            sl = slice(off[c], off[c + 1])
            E0 = O.energy(m[sl], x[sl], v[sl], 1e-3)[2]
            xo, vo, _, _ = O.hermite_shared(m[sl], x[sl], v[sl], 1e-3, 8, steps)
            dE_orc.append(abs(O.energy(m[sl], xo, vo, 1e-3)[2] - E0) / abs(E0))
        dE_orc = np.array(dE_orc)
        ok = dE_gpu[ec] <= 2 * np.maximum(dE_orc, 1e-10)
        out[prec] = {"acc_max_ei": float(max(ea)), "jerk_max_ei": float(max(ej)),
                     "acc_norm_max": float(max(na)), "jerk_norm_max": float(max(nj)),
                     "acc_cond_max": float(max(ca)),
                     "dE_over_E_median_gpu": float(np.median(dE_gpu[ec])),
                     "dE_over_E_median_oracle": float(np.median(dE_orc)),
                     "energy_pass_fraction": float(np.mean(ok)),
                     "dE_ratio_gpu_over_oracle_median": float(np.median(
                         dE_gpu[ec] / np.maximum(dE_orc, 1e-300)))}
    out["sample"] = (f"first evaluation of {n_force} random clusters (seed 2004); energy over "
                     f"{steps} steps of 1/256 from the initial state on {n_energy} of them")
    return out


def run_batched(args):
    """4096 Plummer clusters of log-uniform size in [16, 1024] (seeds
    (1004, c)), eps = 1e-3, shared dt = 1/256, 1000 steps: the persistent
    kernel under a CUDA graph (autotuned shape) against one launch per
    cluster, FP32 and DS."""
    import torch

    from paper_0909_0879_gb300 import _lib, tune

    sizes = ics.cluster_sizes(4096, 1004)
    parts = [ics.plummer(int(nc), (1004, c)) for c, nc in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    m = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    inter = float((sizes.astype(np.float64) ** 2).sum())
    steps = args.batched_steps
    out = {"metric": f"G pair-interactions/s (acc+jerk, 4096 clusters, {steps} shared steps)",
           "unit": UNIT, "workload": f"plummer_clusters_4096_n16-1024_eps1e-3_dt2^-8_{steps}steps",
           "sum_n": int(off[-1]), "sum_n2": inter, "results": {}}
    tuned = {}
    for prec in args.precisions.split(","):
        with _lib.Batch(off, m, x, v, eps=1e-3, lev_shared=8, precision=prec) as b:
            if args.variant >= 0:
                best = (args.variant, steps)
                b.set_tuning(args.variant, steps, 0, True)
            else:
                best, timings = tune.tune_batched(b, steps=20)
            k0, w0 = b.energy()
            b.run(steps)  # capture + warm
            b.sync()
            e0, e1 = _events(torch)
            l0 = b.launch_count()
            e0.record()
            b.run(steps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            launches = b.launch_count() - l0
            k1, w1 = b.energy()
            dE = np.abs((k1 + w1) - (k0 + w0)) / np.abs(k0 + w0)
            # one launch per cluster and step chunk, timed over a few steps
            b.set_tuning(best[0], 1, 0, False)
            pc_steps = 5
            b.run_per_cluster(1)
            b.sync()
            e2, e3 = _events(torch)
            e2.record()
            b.run_per_cluster(pc_steps)
            e3.record()
            torch.cuda.synchronize()
            pc_ms = e2.elapsed_time(e3)
        tuned[prec] = (best[0], best[1])
        out["results"][prec] = {
            "value": inter * steps / ms / 1e6, "ms": ms, "launches": launches,
            "tuned": {"variant": best[0], "steps_per_launch": best[1]},
            "per_cluster_launches": {"value": inter * pc_steps / pc_ms / 1e6, "steps": pc_steps,
                                     "ms": pc_ms},
            f"dE_over_E_median_after_{2 * steps}_steps": float(np.median(dE)),
            "note": "dt = 1/256 with eps = 1e-3 does not resolve close encounters in small "
                    "clusters; the FP64 oracle loses energy at the same level"}
    if not args.no_cpu:
        from oracle import oracle as O

        out["oracle_checks"] = batched_oracle_checks(_lib, O, off, m, x, v, tuned, steps)
        # the oracle's shared-step loop over clusters until ~4e8 interactions
        take, work = [], 0.0
        for c in range(len(sizes)):
            take.append(c)
            work += 16.0 * float(sizes[c]) ** 2
            if work >= 4e8:
                break

        def run_clusters():
            for c in take:
                a, b_ = off[c], off[c + 1]
                O.hermite_shared(m[a:b_], x[a:b_], v[a:b_], 1e-3, 8, 16)

        out["cpu_baseline"] = _oracle_beside(
            run_clusters, work / 1e9, UNIT,
            f"the FP64 oracle's shared-step Hermite loop, 16 steps of the first {len(take)} "
            "clusters")
    print(json.dumps(out), flush=True)
    return 0


def run_adjoint(args):
    """N = 4096 Plummer (seed 1005), eps = 1e-3, 64 KDK steps of dt = 1/128
    in FP32, checkpoints every 8 steps, L = sum |x(T) - y|^2: forward time,
    forward + backward time and buffer memory."""
    import torch

    from paper_0909_0879_gb300 import _lib
    from paper_0909_0879_gb300.autograd import leapfrog

    n, eps, dt, steps, ck = 4096, 1e-3, 1.0 / 128, 64, 8
    m, x, v = ics.plummer(n, 1005)
    y = torch.tensor(x + np.random.default_rng(5).normal(0.0, 0.05, x.shape),
                     dtype=torch.float32, device="cuda")
    x0 = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    v0 = torch.tensor(v, dtype=torch.float32, device="cuda", requires_grad=True)
    mm = torch.tensor(m, dtype=torch.float32, device="cuda", requires_grad=True)
    fwd, both = [], []
    for rep in range(4):
        e0, e1 = _events(torch)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record()
        xT, vT = leapfrog(x0, v0, mm, steps, dt, eps, ckpt_every=ck)
        loss = ((xT - y) ** 2).sum()
        e1.record()
        loss.backward()
        e2.record()
        torch.cuda.synchronize()
        if rep:
            fwd.append(e0.elapsed_time(e1))
            both.append(e0.elapsed_time(e2))
        for t in (x0, v0, mm):
            t.grad = None
    per_eval = n * n
    evals_fwd = steps + 1
    out = {"metric": "ms per forward and forward+backward (leapfrog adjoint, N=4096)",
           "unit": "ms", "workload": "plummer_n4096_eps1e-3_kdk_dt2^-7_64steps_ckpt8",
           "forward_ms": float(np.median(fwd)), "forward_backward_ms": float(np.median(both)),
           "ratio": float(np.median(both) / np.median(fwd)),
           "forward_ginter_s": evals_fwd * per_eval / np.median(fwd) / 1e6,
           "checkpoint_bytes": 4 * _lib.lf_ckpt_floats(n, steps, ck),
           "work_bytes": 4 * _lib.lf_work_floats(n, ck),
           "full_tape_bytes_for_comparison": 4 * (steps + 1) * 6 * n}
    if not args.no_cpu:
        from oracle import oracle as O

        yh = y.double().cpu().numpy()
        cb = _oracle_beside(lambda: O.leapfrog_loss_grad(m, x, v, yh, eps, dt, steps), 1.0,
                            "forward+backward/s",
                            "the FP64 oracle's loss and exact adjoint gradient, same 64 steps")
        cb["forward_backward_ms"] = cb["seconds"] * 1e3
        out["cpu_baseline"] = cb
    print(json.dumps(out), flush=True)
    return 0


def _time_symplectic(torch, s, order, dt, steps):
    """Seconds per step of s.symplectic: the difference of a 0-step call
    (which only evaluates the acceleration at the start) and a `steps`
    call, so each step carries exactly its own force evaluations (and, in
    a spatial layout, the run's share of its ordering).  A first call of
    the same length captures the step's graph."""
    s.symplectic(order, dt, steps)
    ms = []
    for k in (0, steps):
        e0, e1 = _events(torch)
        e0.record()
        s.symplectic(order, dt, k)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return (ms[1] - ms[0]) / 1e3 / steps


def run_symplectic(args):
    """The paper's symplectic integrators (Sec. 2.2) on its own test system
    (Sec. 3): N = 65536 uniform sphere of radius 1, Salpeter masses, virial
    ratio Q = 1, G = M = 1, eps = 0.1 (4 pi / 3 N)^(1/3).
    Speed: per precision, particle layout and order, seconds per step and
    interactions/s over 16 steps (CUDA events; the force evaluation a call
    makes at its start is excluded); layouts are generation order (as the
    paper's particles come) and nb_spatial_order (balanced bisection, which
    lets the split-precision kernel take its tile-relative far field).
    Accuracy (split precision, generation order): relative energy error at
    t = 1/8 at equal force evaluations, sixth order with dt = 2^-7..2^-10
    against the leapfrog with dt / 7.  Galactic field (Sec. 2.1): a cluster
    of N particles on a circular orbit at 8.5 kpc in Allen & Santillan's
    field, energy error in both precisions and the field's cost."""
    import torch

    from paper_0909_0879_gb300 import _lib, metrics

    n = args.n if args.n != N_DEFAULT else 65536
    m, x, v = ics.uniform_sphere(n, 1006, Q=1.0, masses=ics.salpeter_masses(n, 1006))
    eps = 0.1 * (4.0 * np.pi / (3.0 * n)) ** (1.0 / 3.0)
    perm = _lib.spatial_order(x, 256)
    layouts = {"generation": (m, x, v), "spatial": (m[perm], x[perm], v[perm])}
    props = torch.cuda.get_device_properties(0)
    peak = metrics.fp32_peak_tflops(props.multi_processor_count, 2070.0) * 1e12
    speed = []
    # input order x the library's layout setting: generation order stepped as
    # given, with the automatic layout (the default), and with the spatial
    # layout forced; and input presorted with nb_spatial_order stepped as given
    cases = (("generation", "as_given"), ("generation", "auto"), ("generation", "spatial"),
             ("spatial", "as_given"))
    for prec in args.precisions.split(","):
        for lay, mode in cases if prec == "ds" else (("generation", "as_given"),):
            mm, xx, vv = layouts[lay]
            for order in (6, 2):
                with _lib.NBody(mm, xx, vv, eps=eps, precision=prec) as s:
                    s.set_symplectic_layout(mode)
                    per_step = _time_symplectic(torch, s, order, 2.0**-8, 16)
                    used = s.last_symplectic_layout()
                stages = 7 if order == 6 else 1
                ips = stages * n * n / per_step
                speed.append({"precision": prec, "input_order": lay, "layout_setting": mode,
                              "layout_used": used, "order": order,
                              "s_per_step": per_step,
                              "ms_per_force_evaluation": per_step / stages * 1e3,
                              "interactions_per_s": ips,
                              "frac_of_fp32_peak": ips * metrics.FLOPS_PER_ACC_INTERACTION / peak})
                print(json.dumps(speed[-1]), file=sys.stderr, flush=True)
    accuracy = []
    for k in (7, 8, 9, 10):
        row = {"dt_order6": 2.0**-k, "dt_order2": 2.0**-k / 7,
               "force_evaluations": 7 * 2 ** (k - 3)}
        for order, dt, steps in ((6, 2.0**-k, 2 ** (k - 3)), (2, 2.0**-k / 7, 7 * 2 ** (k - 3))):
            with _lib.NBody(m, x, v, eps=eps, precision="ds") as s:
                E0 = s.energy()[2]
                s.symplectic(order, dt, steps)
                row[f"dE_over_E_order{order}"] = abs(s.energy()[2] / E0 - 1.0)
        accuracy.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    # The paper's configuration (Sec. 2.1): a cluster orbiting in the Galactic
    # field of Allen & Santillan (kpc, 2.32e7 solar masses, 10 km/s): Plummer,
    # 1e5 solar masses, virial radius 10 pc, eps = 0.1 pc, on the circular
    # orbit through (8.5, 0, 0); sixth order to t = 1/32 (two crossing times)
    # with dt = 2^-10 and 2^-12; the energy change (with the field's) over the
    # cluster's pair potential energy in both precisions, the step time with
    # and without the field, and 2000 Hermite block steps with and without
    # it.
    mc, xc, vc = ics.plummer(n, 1007)
    Mc, Lc = 0.00431, 0.01
    mc, xc, vc = (mc * Mc, xc * Lc + np.array([8.5, 0.0, 0.0]),
                  vc * np.sqrt(Mc / Lc) + np.array([0.0, 22.0, 0.0]))
    galactic = []
    for prec in args.precisions.split(","):
        row = {"precision": prec}
        for k in (10, 12):
            # energy change to t = 1/32 relative to the cluster's own pair
            # potential energy (the total is dominated by the field's)
            with _lib.NBody(mc, xc, vc, eps=1e-4, precision=prec) as s:
                w_pair = s.energy()[1]
                s.set_external({})
                E0 = s.energy()[2]
                s.symplectic(6, 2.0**-k, 2 ** (k - 5))
                row[f"dE_over_W_pair_dt2^-{k}"] = abs((s.energy()[2] - E0) / w_pair)
        for field in (True, False):
            with _lib.NBody(mc, xc, vc, eps=1e-4, precision=prec) as s:
                if field:
                    s.set_external({})
                per_step = _time_symplectic(torch, s, 6, 2.0**-10, 16)
            row["s_per_step_with_field" if field else "s_per_step_without_field"] = per_step
        # Hermite block steps (device-resident, eta = 0.01, levels 8..20) of
        # the same cluster, 2000 block steps, with and without the field
        for field in (True, False):
            with _lib.NBody(mc, xc, vc, eps=1e-4, precision=prec, eta=0.01, lev_min=8,
                            lev_max=20) as s:
                if field:
                    s.set_external({})
                c0 = s.counters()["interactions"]
                e0, e1 = _events(torch)
                e0.record()
                done, _ = s.run_blocks(1.0, max_blocks=2000)
                e1.record()
                torch.cuda.synchronize()
                inter = s.counters()["interactions"] - c0
            key = "hermite_blocks_with_field" if field else "hermite_blocks_without_field"
            row[key] = {"block_steps": done, "ms": e0.elapsed_time(e1),
                        "interactions_per_s": inter / (e0.elapsed_time(e1) / 1e3)}
        galactic.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"metric": "interactions/s and energy error of the symplectic integrators",
           "unit": "interactions/s", "workload": f"uniform_sphere_salpeter_q1_n{n}_eps0.1d",
           "flops_per_interaction": metrics.FLOPS_PER_ACC_INTERACTION,
           "peak_basis": "FP32 lanes x 2 x 2070 MHz", "speed": speed,
           "energy_at_t_1/8": accuracy,
           "galactic_cluster": {"workload": f"plummer_n{n}_1e5msun_rv10pc_at_8.5kpc_allen_santillan",
                                "rows": galactic}}
    if not args.no_cpu:
        from oracle import oracle as O

        # the acceleration the integrator used, against the FP64 oracle: one
        # sixth-order step (automatic layout), then the stored a = A(x) on
        # 1024 sampled particles
        samp = np.sort(np.random.default_rng(2006).choice(n, 1024, replace=False))
        ferr = {}
        for prec in args.precisions.split(","):
            with _lib.NBody(m, x, v, eps=eps, precision=prec) as s:
                s.symplectic(6, 2.0**-8, 1)
                st = s.get_state(want=("x", "v", "a"))
            ra, rj = O.force_jerk(m, st["x"], st["v"], eps, idx=samp)
            ca, _ = O.force_jerk_abs(m, st["x"], st["v"], eps, idx=samp)
            e = force_error(st["a"][samp], rj, ra, rj, (ca, ca))
            ferr[prec] = {k: e[k] for k in ("acc_max_ei", "acc_p99_ei", "acc_norm",
                                            "acc_cond_max")}
        ferr["sample"] = ("1024 random particles (seed 2006) after one sixth-order step of "
                          "2^-8: the stored acceleration against the oracle's at the same "
                          "positions")
        out["force_err"] = ferr
        out["cpu_baseline"] = _oracle_beside(
            lambda: O.acc(m, x, eps), n * n / 1e9, UNIT,
            "one FP64 acceleration evaluation of all N particles by the oracle (the "
            "symplectic integrators' force)")
    print(json.dumps(out), flush=True)
    return 0


def run_nsweep(args):
    """Seconds per integration step against N on the paper's own test system
    (Sec. 3): uniform sphere of radius 1, Salpeter mass spectrum, velocities
    rescaled to virial ratio Q = 1, G = M = R = 1, eps = 0.1 of the mean
    interparticle distance (4 pi / 3 N)^(1/3).  The quantity of the paper's
    Fig. 1 for this GPU: a Hermite step (all particles, shared dt, acc + jerk)
    in split precision and in FP32, a sixth-order symplectic step (seven
    acceleration-only evaluations, split precision) and a KDK leapfrog step
    of the differentiable FP32 path (acceleration only).  CPU baseline: the FP64 oracle's force + jerk on a bounded
    sample of i-particles against all N, scaled to N, on every host core and
    on one (the paper's OpenMP and serial versions)."""
    import torch

    from oracle import oracle as O
    from paper_0909_0879_gb300 import _lib

    O.build()
    cores = O.max_threads()
    dev = torch.device("cuda", 0)
    k_max = int(np.log2(args.n)) if args.n != N_DEFAULT else 20
    rows = []
    for k in range(10, k_max + 1):
        n = 1 << k
        m, x, v = ics.uniform_sphere(n, 1006, Q=1.0, masses=ics.salpeter_masses(n, 1006))
        eps = 0.1 * (4.0 * np.pi / (3.0 * n)) ** (1.0 / 3.0)
        steps = int(min(20, max(2, 2e10 / (n * n))))
        row = {"n": n, "eps": eps, "gpu_steps_timed": steps}
        for prec in ("ds", "fp32"):
            with _lib.NBody(m, x, v, eps=eps, precision=prec, block_steps=False,
                            lev_shared=10) as s:
                s.step()
                e0, e1 = _events(torch)
                e0.record()
                for _ in range(steps):
                    s.step()
                e1.record()
                torch.cuda.synchronize()
                row[f"hermite_{prec}_s"] = e0.elapsed_time(e1) / 1e3 / steps
        # the same shared steps device-resident (graph replays, no host
        # round trip per step)
        with _lib.NBody(m, x, v, eps=eps, precision="ds", block_steps=False,
                        lev_shared=10) as s:
            s.run_blocks(2.0**-10)
            e0, e1 = _events(torch)
            e0.record()
            done, _ = s.run_blocks((1 + steps) * 2.0**-10)
            e1.record()
            torch.cuda.synchronize()
            row["hermite_ds_device_resident_s"] = e0.elapsed_time(e1) / 1e3 / max(done, 1)
        with _lib.NBody(m, x, v, eps=eps, precision="ds") as s:
            row["symplectic6_ds_s"] = _time_symplectic(torch, s, 6, 2.0**-10, steps)
        fm = torch.tensor(m, dtype=torch.float32, device=dev)
        fx = torch.tensor(x, dtype=torch.float32, device=dev)
        fv = torch.tensor(v, dtype=torch.float32, device=dev)
        fa = torch.empty_like(fx)
        _lib.lf_forward(n, fm, fx, fv, fa, 1, 2.0**-10, None, eps=eps)
        # a forward call starts with one force evaluation before its first
        # step: time a call of 0 steps and one of `steps`, and divide the
        # difference, so each step carries exactly its one evaluation
        ms = []
        for k in (0, steps):
            e0, e1 = _events(torch)
            e0.record()
            _lib.lf_forward(n, fm, fx, fv, fa, k, 2.0**-10, None, eps=eps)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        row["leapfrog_fp32_s"] = (ms[1] - ms[0]) / 1e3 / steps
        # CPU baseline: oracle force + jerk per i-particle, about 0.5 s a point
        rng = np.random.default_rng(8)
        for threads in (cores, 1):
            O.set_threads(threads)
            probe = np.sort(rng.choice(n, min(n, 16), replace=False))
            t0 = time.perf_counter()
            O.force_jerk(m, x, v, eps, idx=probe)
            per_i = (time.perf_counter() - t0) / len(probe)
            ns = int(min(n, max(len(probe), 0.5 / max(per_i, 1e-9))))
            sample = np.sort(rng.choice(n, ns, replace=False))
            t0 = time.perf_counter()
            O.force_jerk(m, x, v, eps, idx=sample)
            dt = time.perf_counter() - t0
            key = "oracle_all_cores_s" if threads == cores else "oracle_1_core_s"
            row[key] = dt * n / ns
            row[key.replace("_s", "_sample")] = ns
        O.set_threads(cores)
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"metric": "seconds per integration step vs N (uniform sphere, Salpeter masses, Q = 1)",
           "unit": "s", "workload": "uniform_sphere_salpeter_q1_eps0.1d", "cores": cores,
           "rows": rows,
           "note": "GPU: CUDA events, all particles stepped each step; oracle: FP64 force + jerk "
                   "on a sample of i-particles against all N, scaled to N (the O(N) part is "
                   "negligible)"}
    print(json.dumps(out), flush=True)
    return 0


def run_isplit(args):
    """The i-split of the paper's two-GPU version (Sec. 4) on one GPU: the
    headline cluster (N = 1,048,576 King W0 = 7 in the spatial layout,
    eps = 1e-4, Hermite shared dt 2^-10, all active) advanced by P shard
    contexts that each evaluate the force and corrector of their slice of
    the active list and exchange the corrected records (one buffer every
    shard exports into and imports from).  Against the unsharded context on
    the same steps: the rate, and the largest position difference."""
    import torch

    from paper_0909_0879_gb300 import _lib, shard

    n, P = args.n, args.shards
    m, x, v = ics.king(n, W0, 1003)
    perm = _lib.spatial_order(x, 256)
    m, x, v = m[perm], x[perm], v[perm]
    kw = dict(eps=EPS, precision=args.precision, block_steps=False, lev_shared=LEV_SHARED)
    out = {"metric": f"G pair-interactions/s (acc+jerk, N={n}, i-split over {P} shards on one "
                     f"GPU)", "unit": UNIT, "workload": workload_name(n), "shards": P,
           "results": {}}
    states = {}
    for name, mk in (("unsharded", lambda: _lib.NBody(m, x, v, **kw)),
                     (f"shards{P}", lambda: shard.ShardGroup(m, x, v, P, **kw))):
        with mk() as g:
            for _ in range(args.warmup):
                g.step()
            torch.cuda.synchronize()
            e0, e1 = _events(torch)
            t0 = time.perf_counter()
            e0.record()
            for _ in range(args.steps):
                g.step()
            e1.record()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            ms = e0.elapsed_time(e1)
            states[name] = g.get_state(want=("x",))["x"]
        out["results"][name] = {"value": args.steps * n * n / ms / 1e6, "ms_per_step":
                                ms / args.steps, "wall_s": wall}
    out["max_abs_dx_vs_unsharded"] = float(np.abs(states[f"shards{P}"] -
                                                  states["unsharded"]).max())
    out["note"] = ("shards run one after another on one GPU (the exchange is a shared buffer); "
                   "on P GPUs each shard's force work is 1/P of the step")
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.workload != "king1m" and args.impl == "ours":
        return {"shared1024": run_shared1024, "block65536": run_block65536,
                "batched": run_batched, "adjoint": run_adjoint,
                "nsweep": run_nsweep, "symplectic": run_symplectic,
                "isplit": run_isplit}[args.workload](args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
