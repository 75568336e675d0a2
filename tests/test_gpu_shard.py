"""i-split shards (the paper's two-GPU version, Sec. 4) on one GPU: P shard
contexts in one process, the all-gather being one record buffer that every
shard exports its slice into.  Each shard evaluates the force and runs the
corrector for its slice of the active list only.  Against the unsharded
context: the same block schedule, and states that differ only by the
rounding of force sums evaluated in other i-block groupings (within the
split-precision force bar carried through the steps); against the FP64
oracle replaying that schedule: positions and energy, as for the unsharded
run."""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu

TICK = 2.0**-20


@pytest.fixture(scope="module")
def nb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    return _lib


@pytest.mark.parametrize("nranks", [2, 3])
def test_shards_follow_unsharded_schedule_and_oracle(nb, oracle_mod, nranks):
    from paper_0909_0879_gb300 import shard

    n, eps, t_end = 1024, 1e-4, 1 << 15  # t = 1/32: every particle synchronised
    m, x, v = ics.plummer(n, 1002, masses=ics.salpeter_masses(n, 1002))
    kw = dict(eps=eps, precision="ds", eta=0.01, eta_start=0.01, lev_min=5, lev_max=20)
    sched_1, sched_p = [], []
    with nb.NBody(m, x, v, **kw) as s:
        lev0 = s.get_state(want=("lev",))["lev"]
        E0 = s.energy()[2]
        while True:
            st = s.get_state(want=("t_tick", "lev"))
            due = st["t_tick"] + (1 << (20 - st["lev"].astype(np.int64)))
            if due.min() > t_end:
                break
            t, na = s.step()
            sched_1.append((int(round(t / TICK)), na))
        ref = s.get_state()
    with shard.ShardGroup(m, x, v, nranks, **kw) as g:
        for s in g.shards:  # identical initial state on every shard
            assert np.array_equal(s.get_state(want=("lev",))["lev"], lev0)
        while True:
            st = g.get_state(want=("t_tick", "lev"))
            due = st["t_tick"] + (1 << (20 - st["lev"].astype(np.int64)))
            if due.min() > t_end:
                break
            t, na = g.step()
            off = g.shards[0].shard_offsets()
            assert off[0] == 0 and off[-1] == na and np.all(np.diff(off) >= 0)
            sched_p.append((int(round(t / TICK)), na))
        states = [s.get_state() for s in g.shards]
        E1 = g.shards[0].energy()[2]
    # the shards agree bit for bit after every import
    for st in states[1:]:
        for k in st:
            assert np.array_equal(st[k], states[0][k]), k
    got = states[0]
    assert sched_p == sched_1, "the sharded run took other block steps"
    assert np.all(got["t_tick"] == t_end)
    assert np.array_equal(got["lev"], ref["lev"])
    # differences of rounding only: force sums agree to ~1e-7 relative, so
    # positions to ~1e-7 |a| T^2
    amag = np.linalg.norm(ref["a"], axis=1)
    T = t_end * TICK
    assert np.all(np.linalg.norm(got["x"] - ref["x"], axis=1) <= 1e-6 * amag * T * T + 1e-12)
    assert np.all(np.linalg.norm(got["v"] - ref["v"], axis=1) <= 1e-6 * amag * T + 1e-12)
    # the FP64 oracle replaying the schedule
    orc = oracle_mod.HermiteState(m, x, v, eps, eta=0.01, eta_start=0.01, lev_min=5, lev_max=20)
    orc.lev[:] = lev0
    E0o = orc.energy()[2]
    with nb.NBody(m, x, v, **kw) as s:
        for tn, na in sched_1:
            t, na2 = s.next_block()
            act = s.active()
            assert int(round(t / TICK)) == tn and na2 == na
            s.predict(t)
            s.force_jerk_dev(None, na, None, None)
            s.correct(t)
            orc.step(replay=(tn, act.astype(np.int64)))
    E1o = orc.energy()[2]
    dE, dEo = abs(E1 - E0) / abs(E0), abs(E1o - E0o) / abs(E0o)
    print(f"P = {nranks}: {len(sched_p)} block steps, dE/E shards {dE:.3e} oracle {dEo:.3e}")
    assert dE <= 2 * max(dEo, 1e-10)
    assert np.abs(got["x"] - orc.x).max() < 1e-6


def test_shard_protocol(nb):
    n = 600
    m, x, v = ics.plummer(n, 3)
    with nb.NBody(m, x, v, eps=1e-3) as s:
        with pytest.raises(nb.NBodyError) as e:
            s.shard_set(2, 0, [0, 100, 500])  # does not end at n
        assert e.value.status == nb.NB_ERR_INVALID_ARG
        with pytest.raises(nb.NBodyError) as e:
            s.shard_set(2, 2, [0, 300, n])  # rank out of range
        assert e.value.status == nb.NB_ERR_INVALID_ARG
        s.shard_set(2, 1, [0, 300, n])
        with pytest.raises(nb.NBodyError) as e:
            s.run_blocks(2.0**-6)
        assert e.value.status == nb.NB_ERR_STATE
        t, na = s.next_block()
        s.predict(t)
        s.force_jerk_dev(None, na, None, None)
        s.correct(t)
        with pytest.raises(nb.NBodyError) as e:
            s.next_block()  # the other shard's records are not imported yet
        assert e.value.status == nb.NB_ERR_STATE
        import torch

        rec = torch.zeros((na, nb.SHARD_RECORD_DOUBLES), dtype=torch.float64, device="cuda")
        off = s.shard_offsets()
        cnt = s.shard_export(rec[int(off[1]):])
        assert cnt == off[2] - off[1]
        with pytest.raises(nb.NBodyError) as e:
            s.shard_import(rec, na + 1)
        assert e.value.status == nb.NB_ERR_INVALID_ARG
        s.shard_import(rec, na)
        s.shard_set(1, 0)
        s.next_block()
