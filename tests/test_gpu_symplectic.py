"""GPU parity of the fixed-step symplectic integrators (the kick-drift-kick
leapfrog and the seven-stage sixth-order composition, Sec. 2.2) against the
FP64 oracle.

Bar.  The GPU integrates the same FP64 state as the oracle; only its forces
differ, by at most tol * sum_j |f_ij| per particle (tol = 1e-6 for split
precision, the force bar; 2e-5 for FP32: about 10 ulps per pair term plus
one per term of the 256-term tile sums and of the per-tile total).  Over a
time T a force error da moves a particle by at most T^2/2 max|da| and
changes its velocity by at most T max|da| (the feedback of the position
error on the force is second order at eps = 0.05, where the largest tidal
rate, m / eps^3 = 8, gives a time scale of 0.35 >> T = 1/8).  The tests
take twice those bounds per particle, and check that the order-2 and
order-6 results differ by far more, so a wrong weight or stage order
cannot pass.
"""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"ds": 1e-6, "fp32": 2e-5}


@pytest.fixture(scope="module")
def nb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    return _lib


def _aabs_max(oracle_mod, m, xs, eps):
    """Per-particle max over the given positions of sum_j |f_ij|."""
    out = None
    for x in xs:
        aabs, _ = oracle_mod.force_jerk_abs(m, x, np.zeros_like(x), eps)
        out = aabs if out is None else np.maximum(out, aabs)
    return out


@pytest.mark.parametrize("prec", ["ds", "fp32"])
def test_symplectic_matches_oracle(nb, oracle_mod, prec):
    """N = 1000 (ragged: 3 tiles + 232) Plummer, eps = 0.05, 4 steps of
    dt = 1/32, orders 2 and 6."""
    n, eps, dt, ns = 1000, 0.05, 1.0 / 32, 4
    T = dt * ns
    m, x, v = ics.plummer(n, 11)
    res = {}
    for order in (2, 6):
        with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
            s.symplectic(order, dt, ns)
            st = s.get_state(want=("x", "v", "a"))
        xo, vo = oracle_mod.symplectic(m, x, v, eps, dt, ns, order)
        aabs = _aabs_max(oracle_mod, m, (x, xo), eps)
        ex = np.linalg.norm(st["x"] - xo, axis=1)
        ev = np.linalg.norm(st["v"] - vo, axis=1)
        bx = T * T * TOL[prec] * aabs
        bv = 2 * T * TOL[prec] * aabs
        print(prec, order, "max dx / bound %.3g, max dv / bound %.3g"
              % ((ex / bx).max(), (ev / bv).max()))
        assert np.all(ex <= bx) and np.all(ev <= bv)
        # the acceleration left in the state is A(x) at the final positions
        ao, _ = oracle_mod.force_jerk(m, st["x"], np.zeros_like(xo), eps)
        cond = np.linalg.norm(st["a"] - ao, axis=1) / _aabs_max(oracle_mod, m, (st["x"],), eps)
        assert cond.max() <= TOL[prec]
        res[order] = (st["x"], bx)
    # the two orders differ by far more than the bound
    d26 = np.linalg.norm(res[2][0] - res[6][0], axis=1)
    assert np.median(d26 / res[6][1]) > 10.0


@pytest.mark.parametrize("prec", ["ds", "fp32"])
@pytest.mark.parametrize("n,eps", [(1000, 1e-3), (70001, 1e-3), (1000, 0.0), (70001, 0.0)])
def test_acceleration_only_kernel_equals_jerk_kernel(nb, oracle_mod, prec, n, eps):
    """nsteps = 0 only evaluates A(x) with the acceleration-only kernel; the
    acceleration sums are the same operations in the same order as those
    of the acceleration + jerk kernel that nb_init ran at the same
    positions with the same shape and grid: bit-identical.  eps = 0 takes
    the masked shapes.  The FP32 long-list case is the exception: there the
    acceleration-only form holds 8 particles per thread instead of 4, which
    groups the sums differently, so it meets the FP32 force bar instead."""
    m, x, v = ics.plummer(n, 12)
    with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
        a0 = s.get_state(want=("a",))["a"]
        s.symplectic(6, 1.0 / 64, 0)
        a1 = s.get_state(want=("a", "x"))
    assert np.array_equal(a1["x"], x)
    if prec == "fp32" and n > 4096 and eps > 0:
        aabs, _ = oracle_mod.force_jerk_abs(m, x, np.zeros_like(x), eps)
        assert np.all(np.linalg.norm(a1["a"] - a0, axis=1) <= 2 * TOL["fp32"] * aabs)
        assert not np.array_equal(a1["a"], a0)
    else:
        assert np.array_equal(a1["a"], a0)


@pytest.mark.parametrize("prec", ["ds", "fp32"])
def test_kepler_two_body_on_gpu(nb, oracle_mod, prec):
    """Two bodies (eps = 0, the masked shapes; n = 2, one padded tile) on an
    e = 0.5 orbit for 1000 sixth-order steps of 2/1000 (graph replayed
    1000 times): the GPU follows the oracle's discrete map within the
    force-error bound and both stay within 1e-6 of Kepler's closed form."""
    import math

    m = np.array([0.5, 0.5])
    rp, vp = 0.5, math.sqrt(3.0)
    x = np.array([[-rp / 2, 0.0, 0.0], [rp / 2, 0.0, 0.0]])
    v = np.array([[0.0, -vp / 2, 0.0], [0.0, vp / 2, 0.0]])
    dt, ns = 2.0 / 1000, 1000
    with nb.NBody(m, x, v, eps=0.0, precision=prec) as s:
        s.symplectic(6, dt, ns)
        st = s.get_state(want=("x",))
    xo, _ = oracle_mod.symplectic(m, x, v, 0.0, dt, ns, 6)
    E = 2.0  # Kepler's equation at t = 2, a = 1, e = 0.5, n = 1
    for _ in range(60):
        E -= (E - 0.5 * math.sin(E) - 2.0) / (1 - 0.5 * math.cos(E))
    rel = np.array([math.cos(E) - 0.5, math.sqrt(0.75) * math.sin(E), 0.0])
    tol = TOL[prec]
    # |a| <= 1 / r_p^2 = 4 along the orbit, T = 2: T^2 tol |a|
    assert np.linalg.norm(st["x"] - xo) <= 4.0 * 4.0 * tol * 4.0
    assert np.linalg.norm((xo[1] - xo[0]) - rel) < 1e-6
    assert np.linalg.norm((st["x"][1] - st["x"][0]) - rel) < 1e-6 + 64 * tol


def test_symplectic6_reversible_on_gpu(nb, oracle_mod):
    """Six steps forward, velocities negated, six steps again: back to the
    start within the force-error bound (a kick merged across the wrong
    stages or a missing closing half kick breaks this by orders of
    magnitude)."""
    n, eps, dt, ns = 1000, 0.05, 1.0 / 32, 6
    T = dt * ns
    m, x, v = ics.plummer(n, 13)
    with nb.NBody(m, x, v, eps=eps, precision="ds") as s:
        s.symplectic(6, dt, ns)
        st = s.get_state()
        st["v"] = -st["v"]
        s.set_state(st)
        s.symplectic(6, dt, ns)
        back = s.get_state(want=("x", "v"))
    aabs = _aabs_max(oracle_mod, m, (x, st["x"]), eps)
    ex = np.linalg.norm(back["x"] - x, axis=1)
    ev = np.linalg.norm(-back["v"] - v, axis=1)
    assert np.all(ex <= 2 * T * T * TOL["ds"] * aabs)
    assert np.all(ev <= 4 * T * TOL["ds"] * aabs)


def test_symplectic_protocol(nb):
    """Bad order / non-finite dt / negative count are rejected; after a
    symplectic run the Hermite calls answer NB_ERR_STATE until set_state;
    a negative dt integrates backwards."""
    m, x, v = ics.plummer(300, 14)
    with nb.NBody(m, x, v, eps=1e-2, precision="ds") as s:
        for args in ((4, 0.01, 1), (6, float("nan"), 1), (2, 0.01, -1)):
            with pytest.raises(nb.NBodyError) as ei:
                s.symplectic(*args)
            assert ei.value.status == 1
        s.symplectic(2, 1.0 / 64, 3)
        with pytest.raises(nb.NBodyError) as ei:
            s.step()
        assert ei.value.status == 2
        with pytest.raises(nb.NBodyError):
            s.run_blocks(1.0)
        st = s.get_state()
        s.symplectic(2, -1.0 / 64, 3)
        back = s.get_state(want=("x",))
        assert np.abs(back["x"] - x).max() < 1e-9
        s.set_state(st)
        s.step()


def test_symplectic6_energy_at_bench_size(nb, oracle_mod):
    """The bench's workload: N = 65536 uniform sphere, Salpeter masses,
    Q = 1, eps = 0.1 of the mean interparticle distance, split precision.
    Properties that hold at any size: the final acceleration matches the
    oracle on 256 sampled particles within the force bar, and at dt = 2^-7
    the sixth-order energy error over 8 steps is below the leapfrog's."""
    n = 65536
    m, x, v = ics.uniform_sphere(n, 1006, Q=1.0, masses=ics.salpeter_masses(n, 1006))
    eps = 0.1 * (4.0 * np.pi / (3.0 * n)) ** (1.0 / 3.0)
    dE = {}
    for order in (2, 6):
        with nb.NBody(m, x, v, eps=eps, precision="ds") as s:
            E0 = s.energy()[2]
            s.symplectic(order, 2.0**-7, 8)
            dE[order] = abs(s.energy()[2] / E0 - 1.0)
            st = s.get_state(want=("x", "a"))
        if order == 6:
            idx = np.sort(np.random.default_rng(3).choice(n, 256, replace=False)).astype(np.int32)
            zv = np.zeros_like(st["x"])
            ao, _ = oracle_mod.force_jerk(m, st["x"], zv, eps, idx=idx)
            aabs, _ = oracle_mod.force_jerk_abs(m, st["x"], zv, eps, idx=idx)
            cond = np.linalg.norm(st["a"][idx] - ao, axis=1) / aabs
            assert cond.max() <= TOL["ds"]
    print("dE/E order 2 %.3e, order 6 %.3e" % (dE[2], dE[6]))
    assert dE[6] < dE[2]


def _cluster_in_galaxy(n, seed):
    """A Plummer cluster of 1e5 solar masses (0.00431 units of 2.32e7) and
    virial radius 10 pc, on the circular orbit through (8.5, 0, 0) kpc of
    the Allen & Santillan field (22 units of 10 km/s)."""
    m, x, v = ics.plummer(n, seed)
    M, L = 0.00431, 0.01
    return m * M, x * L + np.array([8.5, 0.0, 0.0]), v * np.sqrt(M / L) + np.array([0.0, 22.0, 0.0])


def test_external_field_cluster_matches_oracle(nb, oracle_mod):
    """The paper's configuration (Sec. 2.1): a star cluster orbiting in the
    Galactic field.  N = 1000, eps = 1e-3 kpc (the closest pairs' orbital
    time, sqrt(eps^3 / m) = 0.015, stays far above the run's 0.004), four
    sixth-order steps of 1e-3 (1/15 of the cluster's crossing time), split
    precision, against
    the oracle with the same field, within the force-error bound; the
    acceleration left in the state is pair sum + field at the final
    positions; the energy includes sum m Phi_ext.  The same run in FP32
    (positions rounded at 8.5 kpc, separations of 1e-3) is far less
    accurate, which is the paper's case for extended precision."""
    n, eps, dt, ns = 1000, 1e-3, 1e-3, 4
    T = dt * ns
    m, x, v = _cluster_in_galaxy(n, 21)
    xo, vo = oracle_mod.symplectic(m, x, v, eps, dt, ns, 6, ext={})
    aabs = _aabs_max(oracle_mod, m, (x, xo), eps)
    errs = {}
    for prec in ("ds", "fp32"):
        with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
            s.set_external({})
            k0, w0, e0 = s.energy()
            s.symplectic(6, dt, ns)
            st = s.get_state(want=("x", "v", "a"))
        ex = np.linalg.norm(st["x"] - xo, axis=1)
        errs[prec] = ex.max()
        if prec != "ds":
            continue
        ev = np.linalg.norm(st["v"] - vo, axis=1)
        print("ds max dx / bound %.3g, dv / bound %.3g"
              % ((ex / (T * T * TOL["ds"] * aabs)).max(), (ev / (2 * T * TOL["ds"] * aabs)).max()))
        assert np.all(ex <= T * T * TOL["ds"] * aabs)
        assert np.all(ev <= 2 * T * TOL["ds"] * aabs)
        zv = np.zeros_like(xo)
        ao = oracle_mod.force_jerk(m, st["x"], zv, eps)[0] + oracle_mod.ext_field(st["x"])[0]
        cond = np.linalg.norm(st["a"] - ao, axis=1) / _aabs_max(oracle_mod, m, (st["x"],), eps)
        assert cond.max() <= TOL["ds"]
        K, W, _ = oracle_mod.energy(m, x, v, eps)
        W_ext = float(np.sum(m * oracle_mod.ext_field(x)[1]))
        assert abs(k0 - K) <= 1e-14 * abs(K)
        assert abs(w0 - (W + W_ext)) <= 1e-12 * abs(W + W_ext)
    print("max position error ds %.3e fp32 %.3e" % (errs["ds"], errs["fp32"]))
    assert errs["fp32"] > 10.0 * errs["ds"]


def test_external_field_protocol(nb):
    """Invalid parameters are rejected and leave the context as it was; a
    symplectic run with the field, then Hermite steps with it after
    set_state, then without it."""
    m, x, v = _cluster_in_galaxy(300, 22)
    with nb.NBody(m, x, v, eps=1e-4, precision="ds") as s:
        a0 = s.get_state(want=("a",))["a"]
        for bad in ({"gamma": 1.0}, {"b_disk": 0.0}, {"m_halo": -1.0}, {"G": float("inf")}):
            with pytest.raises(nb.NBodyError) as ei:
                s.set_external(bad)
            assert ei.value.status == 1
        assert np.array_equal(s.get_state(want=("a",))["a"], a0)
        s.set_external({})
        st = s.get_state()
        s.symplectic(6, 1e-3, 2)
        s.set_state(st)
        s.step()
        s.set_external(None)
        s.step()


@pytest.mark.parametrize("prec", ["ds", "fp32"])
def test_spatial_layout_matches_oracle(nb, oracle_mod, prec):
    """The spatial layout (state gathered into a bisection order, stepped,
    scattered back) within the same force-error bound as the particles' own
    order, with x, v and a returned in the caller's order."""
    n, eps, dt, ns = 1000, 0.05, 1.0 / 32, 4
    T = dt * ns
    m, x, v = ics.plummer(n, 11)
    with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
        s.set_symplectic_layout("spatial")
        s.symplectic(6, dt, ns)
        assert s.last_symplectic_layout() == "spatial"
        st = s.get_state(want=("x", "v", "a"))
    xo, vo = oracle_mod.symplectic(m, x, v, eps, dt, ns, 6)
    aabs = _aabs_max(oracle_mod, m, (x, xo), eps)
    assert np.all(np.linalg.norm(st["x"] - xo, axis=1) <= T * T * TOL[prec] * aabs)
    assert np.all(np.linalg.norm(st["v"] - vo, axis=1) <= 2 * T * TOL[prec] * aabs)
    ao, _ = oracle_mod.force_jerk(m, st["x"], np.zeros_like(xo), eps)
    cond = np.linalg.norm(st["a"] - ao, axis=1) / _aabs_max(oracle_mod, m, (st["x"],), eps)
    assert cond.max() <= TOL[prec]


def test_automatic_layout_choice(nb):
    """Automatic layout: the particles' own order for FP32, for zero steps
    and for short split-precision runs; the spatial order for long ones;
    both orders agree to rounding of the force sums."""
    n = 131072
    m, x, v = ics.uniform_sphere(n, 1006, Q=1.0, masses=ics.salpeter_masses(n, 1006))
    eps = 0.1 * (4.0 * np.pi / (3.0 * n)) ** (1.0 / 3.0)
    with nb.NBody(m, x, v, eps=eps, precision="fp32") as s:
        s.symplectic(2, 2.0**-10, 40)
        assert s.last_symplectic_layout() == "as_given"
    res = {}
    for mode in ("auto", "as_given"):
        with nb.NBody(m, x, v, eps=eps, precision="ds") as s:
            s.set_symplectic_layout(mode)
            s.symplectic(2, 2.0**-10, 0)
            assert s.last_symplectic_layout() == "as_given"
            s.symplectic(2, 2.0**-10, 2)
            assert s.last_symplectic_layout() == "as_given"
            s.symplectic(2, 2.0**-10, 40)
            res[mode] = (s.last_symplectic_layout(), s.get_state(want=("x", "v")))
    assert res["auto"][0] == "spatial" and res["as_given"][0] == "as_given"
    xa, xg = res["auto"][1]["x"], res["as_given"][1]["x"]
    assert not np.array_equal(xa, xg)
    assert np.abs(xa - xg).max() < 1e-6  # a misplaced particle would differ by O(0.1)
    with nb.NBody(m, x, v, eps=eps) as s:
        with pytest.raises(KeyError):
            s.set_symplectic_layout("diagonal")
