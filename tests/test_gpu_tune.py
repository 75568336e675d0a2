"""The autotuner (paper_0909_0879_gb300/tune.py) on the GPU.

Force kernel: the tuned table (shape and persistent-grid cap, i.e. the
stream-K j-split, per active-list length) must reproduce the FP64 oracle
within the split-precision bar, and must be no slower than the built-in
choice at each tuned length (it has the built-in shape at the full grid
among its candidates; a 15 % + 20 us margin covers timing noise).

Batched kernel: the tuned (shape, steps per launch) must be one of the
candidates, give oracle-accurate positions, and be no slower than the
built-in setting beyond noise.
"""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    return _lib


def _median_ms(torch, fn, reps=7):
    from paper_0909_0879_gb300 import tune

    return tune._time_ms(fn, reps, flush=True)


def test_tune_force_table_matches_oracle_and_is_not_slower(nb, oracle_mod):
    import torch

    from paper_0909_0879_gb300 import tune

    n, eps = 20000, 1e-4
    m, x, v = ics.plummer(n, 61, masses=ics.salpeter_masses(n, 61))
    dev = torch.device("cuda", 0)
    fractions = (1.0, 1 / 64)
    with nb.NBody(m, x, v, eps=eps, precision="ds") as s:
        table, timings = tune.tune_force(s, fractions=fractions, use_cache=False)
        assert len(table) == 2
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        for _, var, cap in table:
            assert nb.variant_info(var)["precision"] == 1
            assert cap in tune.grid_caps(nsm)
        # every candidate of each length was timed at the full grid
        assert sum(1 for k in timings if k.endswith(":0")) >= 2 * 10
        for f in fractions:
            na = max(1, int(round(n * f)))
            idx = ics.random_active_subset(n, na, 7)
            acc, jerk = s.force_jerk(idx)  # through the installed table
            ra, rj = oracle_mod.force_jerk(m, x, v, eps, idx=idx)
            ca, cj = oracle_mod.force_jerk_abs(m, x, v, eps, idx=idx)
            assert np.linalg.norm(acc - ra) / np.linalg.norm(ra) <= 1e-6
            assert (np.linalg.norm(acc - ra, axis=1) / ca).max() <= 1e-6
            assert np.linalg.norm(jerk - rj) / np.linalg.norm(rj) <= 1e-5
            assert (np.linalg.norm(jerk - rj, axis=1) / cj).max() <= 1e-5
            d_idx = torch.from_numpy(idx).to(dev)
            d_a = torch.empty((na, 3), dtype=torch.float64, device=dev)
            d_j = torch.empty_like(d_a)
            call = lambda: s.force_jerk_dev(d_idx, na, d_a, d_j)  # noqa: E731
            call()
            t_tuned = _median_ms(torch, call)
            s.set_force_table([])
            call()
            t_builtin = _median_ms(torch, call)
            s.set_force_table(table)
            print(f"n_act {na}: tuned {t_tuned:.4f} ms, built-in {t_builtin:.4f} ms, "
                  f"table {table}")
            assert t_tuned <= 1.15 * t_builtin + 0.02


def test_tune_batched_small_set(nb, oracle_mod):
    import torch

    from paper_0909_0879_gb300 import tune

    sizes = ics.cluster_sizes(40, 77, 16, 256)
    ms, xs, vs = [], [], []
    for c, nc in enumerate(sizes):
        m, x, v = ics.plummer(int(nc), (77, c))
        ms.append(m), xs.append(x), vs.append(v)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    m, x, v = np.concatenate(ms), np.concatenate(xs), np.concatenate(vs)
    eps, lev = 1e-3, 8
    with nb.Batch(off, m, x, v, eps=eps, lev_shared=lev) as b:
        best, timings = tune.tune_batched(b, steps=8, spl=(8, 4), use_cache=False)
    assert f"{best[0]}:{best[1]}" in timings
    assert timings[f"{best[0]}:{best[1]}"] == min(timings.values())
    info = nb.batched_variant_info(best[0])
    assert info["precision"] == 1
    steps = 10
    with nb.Batch(off, m, x, v, eps=eps, lev_shared=lev) as b:
        b.set_tuning(best[0], best[1], 0, True)
        b.run(steps)
        st = b.get_state()
    for c in range(len(off) - 1):
        s = slice(off[c], off[c + 1])
        xo, _, ao, _ = oracle_mod.hermite_shared(m[s], x[s], v[s], eps, lev, steps)
        tol = 1e-5 * np.linalg.norm(ao, axis=1) * (steps * 2.0**-lev) ** 2 / 2 + 1e-12
        assert np.all(np.linalg.norm(st["x"][s] - xo, axis=1) <= tol), c
    # no slower than the built-in setting (same step count per timing)
    res = {}
    for name, tun in (("tuned", (best[0], best[1])), ("builtin", (-1, 1000))):
        with nb.Batch(off, m, x, v, eps=eps, lev_shared=lev) as b:
            b.set_tuning(tun[0], tun[1], 0, True)
            b.run(16)
            res[name] = tune._time_ms(lambda: b.run(16), 5)
    print("batched tuned", best, res)
    assert res["tuned"] <= 1.3 * res["builtin"] + 0.05
