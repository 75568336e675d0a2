"""Host-side counting conventions for the throughput metric.

An interaction is one (i, j) evaluation of the softened pair acceleration
and jerk for an active i-particle; a force evaluation over n_act active
particles against n particles counts n_act * n interactions (the i == j
self term included, which the kernels evaluate and which contributes
exactly zero for eps > 0).

FLOPS_PER_INTERACTION = 44 is the per-interaction count used for the FP32
roofline: 6 FADD (position and velocity differences), 3 FFMA (s^2),
1 reciprocal square root, about 5 FMUL, 3 FFMA (d.w), 3 FFMA (acceleration)
and 6 FFMA (jerk), with a fused multiply-add counted as 2 flops and the
reciprocal square root as 1.  The split-precision variant executes extra
additions for the position differences and the per-tile folds; those are
overhead, not algorithmic work, and are not counted.

The paper's own cost model (Sec. 2, Table 1) is about 30 flops per
symmetric acceleration-only pair, n_f = 30 N (N - 1) / 2.
"""
from __future__ import annotations

FLOPS_PER_INTERACTION = 44
# Acceleration only (the symplectic integrators): 3 FADD (differences),
# 3 FFMA (s^2), 1 reciprocal square root, 3 FMUL (1/s^2, m/s, m/s^3) and
# 3 FFMA (acceleration), a fused multiply-add counted as 2 flops.
FLOPS_PER_ACC_INTERACTION = 19
FLOPS_PER_INTERACTION_CONVENTION = 60  # common acc+jerk convention in the literature
PAPER_FLOPS_PER_PAIR = 30
FP32_LANES_PER_SM = 128


def pair_count(n: float) -> float:
    """Distinct unordered pairs among n bodies, N (N - 1) / 2."""
    return n * (n - 1) / 2.0


def interactions(n_act: int, n: int) -> int:
    """Interactions of one force + jerk evaluation: n_act * n."""
    return int(n_act) * int(n)


def fp32_peak_tflops(n_sm: int, sm_mhz: float) -> float:
    """FP32 peak in TFLOP/s: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return n_sm * FP32_LANES_PER_SM * 2.0 * sm_mhz * 1e6 / 1e12


def aggregate_throughput(local_seconds: float, local_units: float, device=None):
    """Whole-job throughput of independent replicas (weak scaling): the
    units every rank processed divided by the slowest rank's time.  Uses
    torch.distributed when initialised (one all-reduce MAX of the time and
    one SUM of the units); otherwise the local values.  Returns
    (units_per_second, max_seconds, total_units)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local_units / local_seconds, local_seconds, local_units
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())
