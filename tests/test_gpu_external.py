"""GPU parity of the Hermite integrator with the external Galactic field
(Allen & Santillan 1991; the paper adds it to the pair forces, Sec. 2.1)
against the FP64 oracle with the same field, and the bit-identity of the
host-driven, general and fused block steps with it.

The field is FP64 on both sides (only the evaluation order of a few
operations differs); the pair forces carry the split-precision force error
(<= 1e-6 of sum_j |f_ij|), which bounds the position and velocity
differences as in the other parity tests."""
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


def _cluster(n, seed):
    """Plummer cluster, 1e5 solar masses (0.00431 units of 2.32e7), virial
    radius 10 pc, on the circular orbit through (8.5, 0, 0) kpc (22 units
    of 10 km/s), Salpeter masses."""
    m, x, v = ics.plummer(n, seed, masses=ics.salpeter_masses(n, seed))
    M, L = 0.00431, 0.01
    return m * M, x * L + np.array([8.5, 0.0, 0.0]), v * np.sqrt(M / L) + np.array([0.0, 22.0, 0.0])


def test_set_external_moves_the_field_into_the_state(nb, oracle_mod):
    """On a fresh context the stored a and jerk become pair sums + field at
    each particle's state and the initial levels are taken from the totals
    (as the oracle's initialisation with the field does); removing the
    field takes it out again."""
    n, eps = 700, 1e-3
    m, x, v = _cluster(n, 31)
    with nb.NBody(m, x, v, eps=eps, precision="ds", eta=0.01, lev_min=6, lev_max=20) as s:
        s0 = s.get_state(want=("a", "jerk", "lev"))
        s.set_external({})
        s1 = s.get_state(want=("a", "jerk", "lev"))
        s.set_external(None)
        s2 = s.get_state(want=("a", "jerk"))
    ea, _, ej = oracle_mod.ext_field(x, v=v)
    assert np.abs(s1["a"] - (s0["a"] + ea)).max() <= 1e-13 * np.abs(ea).max()
    assert np.abs(s1["jerk"] - (s0["jerk"] + ej)).max() <= 1e-13 * np.abs(ej).max()
    assert np.abs(s2["a"] - s0["a"]).max() <= 1e-13 * np.abs(ea).max()
    orc = oracle_mod.HermiteState(m, x, v, eps, eta=0.01, lev_min=6, lev_max=20, ext={})
    assert np.mean(s1["lev"] == orc.lev) > 0.99
    assert not np.array_equal(s1["lev"], s0["lev"])


def test_hermite_shared_steps_in_field_match_oracle(nb, oracle_mod):
    """Shared steps of 2^-12 (1/60 of the cluster's crossing time), 16
    steps, split precision: positions and velocities within the bound set
    by the pair-force error, and the field's share in the stored totals."""
    n, eps, lev, ns = 1000, 1e-3, 12, 16
    T = ns * 2.0**-lev
    m, x, v = _cluster(n, 32)
    xo, vo, ao, jo = oracle_mod.hermite_shared(m, x, v, eps, lev, ns, ext={})
    with nb.NBody(m, x, v, eps=eps, precision="ds", block_steps=False, lev_shared=lev) as s:
        s.set_external({})
        for _ in range(ns):
            s.step()
        st = s.get_state(want=("x", "v", "a", "jerk", "t_tick"))
    assert np.all(st["t_tick"] == ns << (20 - lev))
    aabs = np.maximum(oracle_mod.force_jerk_abs(m, x, v, eps)[0],
                      oracle_mod.force_jerk_abs(m, xo, vo, eps)[0])
    ex = np.linalg.norm(st["x"] - xo, axis=1)
    ev = np.linalg.norm(st["v"] - vo, axis=1)
    print("max dx / bound %.3g, dv / bound %.3g"
          % ((ex / (T * T * 1e-6 * aabs)).max(), (ev / (2 * T * 1e-6 * aabs)).max()))
    assert np.all(ex <= T * T * 1e-6 * aabs)
    assert np.all(ev <= 2 * T * 1e-6 * aabs)
    # the stored acceleration is the total; the field dominates it here
    assert np.all(np.linalg.norm(st["a"] - ao, axis=1) <= 2e-6 * aabs)
    assert np.abs(ao).max() > 50.0


def test_block_steps_in_field_against_oracle(nb, oracle_mod):
    """Aarseth block steps (eta = 0.01, levels 8..20) of the cluster in the
    field to t = 2^-8: the oracle replays the GPU's schedule; positions and
    the energy change (with the field's potential) agree."""
    n, eps = 1024, 1e-3
    t_end = 1 << 12  # 2^-8 in ticks
    m, x, v = _cluster(n, 33)
    with nb.NBody(m, x, v, eps=eps, precision="ds", eta=0.01, lev_min=8, lev_max=20) as s:
        s.set_external({})
        lev0 = s.get_state(want=("lev",))["lev"]
        orc = oracle_mod.HermiteState(m, x, v, eps, eta=0.01, lev_min=8, lev_max=20, ext={})
        assert np.mean(lev0 == orc.lev) > 0.99
        orc.lev[:] = lev0
        E0 = s.energy()[2]
        sched = []
        while True:
            st = s.get_state(want=("t_tick", "lev"))
            due = st["t_tick"] + (1 << (20 - st["lev"].astype(np.int64)))
            if due.min() > t_end:
                break
            t, na = s.next_block()
            act = s.active().astype(np.int64)
            s.predict(t)
            s.force_jerk_dev(None, na, None, None)
            s.correct(t)
            sched.append((int(round(t / TICK)), act))
        stg = s.get_state()
        E1 = s.energy()[2]
    assert np.all(stg["t_tick"] == t_end)
    E0o = orc.energy()[2]
    for tn, act in sched:
        orc.step(replay=(tn, act))
    E1o = orc.energy()[2]
    print("block steps", len(sched), "dE gpu %.3e oracle %.3e" % (E1 - E0, E1o - E0o))
    assert abs(E0 - E0o) <= 1e-12 * abs(E0o)
    # energy changes against the cluster's own binding energy (the field's
    # potential dominates the total)
    W = abs(oracle_mod.energy(m, x, v, eps)[1])
    assert abs((E1 - E0) - (E1o - E0o)) <= 1e-6 * W
    assert np.abs(stg["x"] - orc.x).max() < 1e-9
    assert np.mean(stg["lev"] == orc.lev) > 0.98


@pytest.mark.parametrize("prec", ["ds", "fp32"])
def test_fused_and_general_block_steps_with_field_match_host(nb, prec):
    """With the field set, the fused device-resident steps, the general
    scheduler and the nb_step loop take the same steps with the same bits;
    changing the field drops the cached graphs."""
    n = 1500 + 33
    m, x, v = _cluster(n, 34)
    kw = dict(eps=1e-3, eta=0.02, lev_min=8, lev_max=20, precision=prec)
    t_end = 2.0**-8
    with nb.NBody(m, x, v, **kw) as a:
        a.set_external({})
        s_init = a.get_state()
        steps = a.run_until(t_end)
        sa = a.get_state()
    for mode in ("auto", "general"):
        with nb.NBody(m, x, v, **kw) as b:
            b.set_block_mode(mode)
            b.run_blocks(2.0**-10)  # graphs captured without the field
            b.set_external({})
            b.set_state(s_init)
            done, t_last = b.run_blocks(t_end)
            assert b.last_block_path() == ("fused" if mode == "auto" else "general")
            sb = b.get_state()
        assert done == steps and t_last == t_end
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), (prec, mode, k)


def test_field_parameters_reach_the_device(nb, oracle_mod):
    """A field with every parameter changed from Allen & Santillan's (centre
    off the origin, other masses, scales, exponent and cut) moves the same
    acceleration and jerk into the state as the oracle computes."""
    ext = {"G": 0.9, "center": (0.4, -0.3, 0.2), "m_bulge": 500.0, "b_bulge": 0.5,
           "m_disk": 3000.0, "a_disk": 4.0, "b_disk": 0.3, "m_halo": 5000.0,
           "a_halo": 10.0, "gamma": 2.2, "r_cut": 9.0}
    n = 500
    m, x, v = _cluster(n, 35)
    x = x + np.array([0.0, 0.0, 0.5])  # off the plane
    with nb.NBody(m, x, v, eps=1e-3, precision="ds") as s:
        s0 = s.get_state(want=("a", "jerk"))
        s.set_external(ext)
        s1 = s.get_state(want=("a", "jerk"))
        _, w, _ = s.energy()
    ea, phi, ej = oracle_mod.ext_field(x, ext, v=v)
    assert np.abs(s1["a"] - s0["a"] - ea).max() <= 1e-12 * np.abs(ea).max()
    assert np.abs(s1["jerk"] - s0["jerk"] - ej).max() <= 1e-12 * np.abs(ej).max()
    W = oracle_mod.energy(m, x, v, 1e-3)[1] + float(np.sum(m * phi))
    assert abs(w - W) <= 1e-12 * abs(W)
