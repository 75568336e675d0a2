"""Pins for the oracle's Hermite-4 block-step integrator and its KDK
leapfrog with adjoint (CPU only)."""
import math

import numpy as np
import pytest

from paper_0909_0879_gb300 import ics


# ----------------------------------------------------------------- Kepler


def kepler_ic(e=0.5, a=1.0, m1=0.5, m2=0.5):
    """Two bodies at pericentre of a relative orbit (semi-major axis a,
    eccentricity e) in the centre-of-mass frame, G = 1."""
    M = m1 + m2
    rp = a * (1 - e)
    vp = math.sqrt(M * (1 + e) / (a * (1 - e)))
    rel_x = np.array([rp, 0.0, 0.0])
    rel_v = np.array([0.0, vp, 0.0])
    m = np.array([m1, m2])
    x = np.array([-m2 / M * rel_x, m1 / M * rel_x])
    v = np.array([-m2 / M * rel_v, m1 / M * rel_v])
    return m, x, v


def kepler_relative_position(t, e=0.5, a=1.0, M=1.0):
    """Kepler's equation E - e sin E = n t solved by Newton's method."""
    n = math.sqrt(M / a**3)
    Mean = n * t
    E = Mean
    for _ in range(60):
        E -= (E - e * math.sin(E) - Mean) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def test_kepler_fourth_order_convergence(oracle_mod):
    """Hermite-4 with shared dt on the eps = 0 two-body problem: the position
    error after ~3 orbits (e = 0.5) against Kepler's equation falls by ~2^4 when dt
    halves."""
    m, x, v = kepler_ic()
    errs = []
    t_end = 20.0
    for lev in (7, 8, 9):
        nsteps = int(t_end * 2**lev)
        xf, vf, _, _ = oracle_mod.hermite_shared(m, x, v, 0.0, lev, nsteps)
        rel = xf[1] - xf[0]
        errs.append(np.linalg.norm(rel - kepler_relative_position(t_end)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, (errs, r1, r2)
    assert errs[2] < 1e-8


def test_kepler_one_step_local_error_sixth_order(oracle_mod):
    """One Hermite step from pericentre: the corrected position reproduces
    the Taylor series through the dt^5 term (a2 dt^4/24 + a3 dt^5/120), so
    its local error falls by ~2^6 per halving of dt."""
    m, x, v = kepler_ic()
    errs = []
    for lev in (5, 6, 7):
        xf, _, _, _ = oracle_mod.hermite_shared(m, x, v, 0.0, lev, 1)
        rel = xf[1] - xf[0]
        errs.append(np.linalg.norm(rel - kepler_relative_position(2.0**-lev)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 56.0 < r1 < 72.0 and 56.0 < r2 < 72.0, (errs, r1, r2)


def test_kepler_invariants(oracle_mod):
    """Energy, angular momentum and the Laplace-Runge-Lenz vector of the
    relative orbit are conserved to the integrator's error level."""
    m, x, v = kepler_ic()
    st = oracle_mod.HermiteState(m, x, v, 0.0, block_levels=False, shared_lev=8)
    E0 = st.energy()[2]

    def lrl(x, v):
        r = x[1] - x[0]
        u = v[1] - v[0]
        L = np.cross(r, u)
        return np.cross(u, L) - r / np.linalg.norm(r), L

    A0, L0 = lrl(st.x, st.v)
    for _ in range(int(2 * math.pi * 256)):
        st.step()
    E1 = st.energy()[2]
    A1, L1 = lrl(st.x, st.v)
    assert abs(E1 - E0) / abs(E0) < 1e-9
    assert np.linalg.norm(L1 - L0) < 1e-9
    assert np.linalg.norm(A1 - A0) < 1e-7
    P = (m[:, None] * st.v).sum(0)
    assert np.linalg.norm(P) < 1e-15


def test_aarseth_criterion_circular_orbit(oracle_mod):
    """Uniform circular motion of radius R and rate w has |a| = w^2 R,
    |j| = w^3 R, |a2| = w^4 R, |a3| = w^5 R, so the criterion gives
    dt = sqrt(eta) / w exactly."""
    R, w, eta = 1.7, 2.3, 0.01
    ph = 0.4
    r = R * np.array([math.cos(ph), math.sin(ph), 0.0])
    u = R * w * np.array([-math.sin(ph), math.cos(ph), 0.0])
    a, jk, a2, a3 = -w**2 * r, -w**2 * u, w**4 * r, w**4 * u
    dt = oracle_mod.aarseth_dt(a, jk, a2, a3, eta)
    assert abs(dt - math.sqrt(eta) / w) < 1e-15


def test_level_quantisation(oracle_mod):
    """dt -> largest power of two not above it, clamped to [3, 20]."""
    L = oracle_mod.level_from_dt
    assert L(0.25) == (2 if False else 3, False)  # 2^-2 clamps to lev_min = 3
    assert L(0.25, 1, 20) == (2, False)
    assert L(0.3, 1, 20) == (2, False)
    assert L(0.2499999, 1, 20) == (3, False)
    assert L(2.0**-20) == (20, False)
    assert L(2.0**-20 * 0.999) == (20, True)
    assert L(1e-9) == (20, True)
    assert L(10.0) == (3, False)
    N = oracle_mod.next_level
    # shrink freely
    assert N(5, 9, 12345) == 9
    # grow one level only, and only on a multiple of the doubled step
    assert N(5, 3, 1 << 16) == 4          # 2^16 ticks is a multiple of 2^(20-4)
    assert N(5, 3, 3 << 15) == 5          # not a multiple of 2^16
    assert N(3, 3, 0) == 3
    assert N(4, 3, 1 << 17, lev_min=4) == 4


def test_block_schedule_invariants_and_sync(oracle_mod):
    """Block steps on a Salpeter-mass Plummer sphere: every t_i stays a
    multiple of its own step, t_next never decreases, the active set is the
    set of particles due at t_next, and every particle lands on t = 1/8."""
    n = 128
    m, x, v = ics.plummer(n, 5, masses=ics.salpeter_masses(n, 5))
    st = oracle_mod.HermiteState(m, x, v, 1e-3, eta=0.02, eta_start=0.01)
    E0 = st.energy()[2]
    t_end = 1 << 17
    t_prev = 0
    steps = 0
    while True:
        due = st.t + (1 << (20 - st.lev.astype(np.int64)))
        if due.min() > t_end:
            break
        tn, act = st.step()
        steps += 1
        assert tn >= t_prev
        t_prev = tn
        assert np.array_equal(act, np.nonzero(due == tn)[0])
        assert np.all(st.t[act] == tn)
        assert np.all(st.t % (1 << (20 - st.lev.astype(np.int64))) == 0)
    assert np.all(st.t == t_end)
    assert steps > 8 and len(np.unique(st.lev)) > 1
    E1 = st.energy()[2]
    assert abs(E1 - E0) / abs(E0) < 1e-5


def test_block_equals_shared_on_uniform_levels(oracle_mod):
    """With the criterion forced to the largest step (huge eta) every
    particle stays at lev_min and the block-step path reproduces the
    shared-step path bit for bit."""
    m, x, v = ics.plummer(64, 8)
    st = oracle_mod.HermiteState(m, x, v, 1e-2, eta=1e12, eta_start=1e12, lev_min=6, lev_max=20)
    assert np.all(st.lev == 6)
    for _ in range(8):
        st.step()
    xs, vs, _, _ = oracle_mod.hermite_shared(m, x, v, 1e-2, 6, 8)
    assert np.array_equal(st.x, xs) and np.array_equal(st.v, vs)


def test_replay_follows_given_schedule(oracle_mod):
    """Replay mode reproduces a free run when fed that run's own schedule."""
    m, x, v = ics.plummer(48, 12)
    a = oracle_mod.HermiteState(m, x, v, 1e-3, eta=0.02)
    b = oracle_mod.HermiteState(m, x, v, 1e-3, eta=0.02)
    for _ in range(30):
        tn, act = a.step()
        b.step(replay=(tn, act))
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)


# --------------------------------------------------------------- leapfrog


def test_leapfrog_time_reversible(oracle_mod):
    m, x, v = ics.plummer(32, 4)
    x1, v1 = oracle_mod.leapfrog(m, x, v, 1e-2, 1 / 128, 40)
    x2, v2 = oracle_mod.leapfrog(m, x1, -v1, 1e-2, 1 / 128, 40)
    assert np.abs(x2 - x).max() < 1e-11 and np.abs(-v2 - v).max() < 1e-11


def test_leapfrog_energy_bounded(oracle_mod):
    """Symplectic: on Kepler the energy error oscillates without secular
    growth (paper Sec. 3.1).  The largest error seen during the last ten of
    twenty orbits is no larger than during the first ten."""
    m, x, v = kepler_ic(e=0.3)
    E0 = oracle_mod.energy(m, x, v, 0.0)[2]
    dt = 1 / 64
    per = int(round(2 * math.pi / dt))
    errs = []
    for _ in range(20 * per):
        x, v = oracle_mod.leapfrog(m, x, v, 0.0, dt, 1)
        errs.append(abs(oracle_mod.energy(m, x, v, 0.0)[2] - E0))
    half = 10 * per
    assert max(errs[half:]) < 1.05 * max(errs[:half])
    assert max(errs) < 1e-3 * abs(E0)


def test_acc_vjp_vs_finite_differences(oracle_mod):
    """d(g . A(x, m))/dx_k and /dm_k by central differences."""
    rng = np.random.default_rng(3)
    n = 10
    m = rng.uniform(0.2, 1.0, n)
    x = rng.normal(0, 1, (n, 3))
    g = rng.normal(0, 1, (n, 3))
    eps = 0.1
    gx, gm = oracle_mod.acc_vjp(m, x, g, eps)
    h = 1e-6

    def f(mm, xx):
        return np.sum(g * oracle_mod.acc(mm, xx, eps))

    for k in range(n):
        for c in range(3):
            xp = x.copy(); xp[k, c] += h
            xm = x.copy(); xm[k, c] -= h
            fd = (f(m, xp) - f(m, xm)) / (2 * h)
            assert abs(fd - gx[k, c]) < 1e-7 * (1 + abs(fd))
        mp_ = m.copy(); mp_[k] += h
        mm_ = m.copy(); mm_[k] -= h
        fd = (f(mp_, x) - f(mm_, x)) / (2 * h)
        assert abs(fd - gm[k]) < 1e-7 * (1 + abs(fd))


def test_leapfrog_adjoint_vs_finite_differences(oracle_mod):
    """Gradient of L = sum |x(T) - y|^2 after KDK steps against FP64 central
    differences on sampled coordinates of x0, v0 and m."""
    n = 24
    m, x, v = ics.plummer(n, 5)
    y = x + np.random.default_rng(5).normal(0, 0.05, x.shape)
    eps, dt, ns = 1e-2, 1 / 128, 16
    L, gx, gv, gm = oracle_mod.leapfrog_loss_grad(m, x, v, y, eps, dt, ns)

    def loss(mm, xx, vv):
        xf, _ = oracle_mod.leapfrog(mm, xx, vv, eps, dt, ns)
        return np.sum((xf - y) ** 2)

    assert abs(loss(m, x, v) - L) < 1e-14 * abs(L)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(12):
        k, c = rng.integers(n), rng.integers(3)
        for arr, grad in ((x, gx), (v, gv)):
            ap = arr.copy(); ap[k, c] += h
            am = arr.copy(); am[k, c] -= h
            if arr is x:
                fd = (loss(m, ap, v) - loss(m, am, v)) / (2 * h)
            else:
                fd = (loss(m, x, ap) - loss(m, x, am)) / (2 * h)
            assert abs(fd - grad[k, c]) < 1e-6 * (abs(fd) + 1e-3 * np.abs(grad).max())
        mp_ = m.copy(); mp_[k] += h * m[k]
        mm_ = m.copy(); mm_[k] -= h * m[k]
        fd = (loss(mp_, x, v) - loss(mm_, x, v)) / (2 * h * m[k])
        assert abs(fd - gm[k]) < 1e-6 * (abs(fd) + 1e-3 * np.abs(gm).max())


def test_leapfrog_adjoint_short_step_limit(oracle_mod):
    """One step with dt -> 0 leaves x unchanged, so dL/dx0 -> 2 (x0 - y)."""
    m, x, v = ics.plummer(16, 2)
    y = x + 0.1
    L, gx, gv, gm = oracle_mod.leapfrog_loss_grad(m, x, v, y, 1e-2, 1e-9, 1)
    assert np.abs(gx - 2 * (x - y)).max() < 1e-7
    assert np.abs(gm).max() < 1e-12


# ------------------------------------------------ sixth-order symplectic


def test_symplectic6_weights_order_conditions(oracle_mod):
    """The seven weights of a symmetric composition of a symmetric
    second-order step reach order 6 only if they sum to 1 (consistency)
    and their third and fifth powers sum to 0 (the h^3 and h^5 error terms
    of the base step cancel); the symmetry w_k = w_{6-k} removes the even
    orders."""
    w = np.array(oracle_mod.SYMPLECTIC6_WEIGHTS)
    assert w.shape == (7,)
    assert np.array_equal(w, w[::-1])
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs(np.sum(w**3)) < 1e-13
    assert abs(np.sum(w**5)) < 1e-13


def _kepler_errors(oracle_mod, order, ks, t_end=2.0, weights=None):
    m, x, v = kepler_ic()
    errs = []
    for k in ks:
        xf, _ = oracle_mod.symplectic(m, x, v, 0.0, t_end / k, k, order, weights=weights)
        errs.append(np.linalg.norm((xf[1] - xf[0]) - kepler_relative_position(t_end)))
    return errs


def test_symplectic_convergence_orders_kepler(oracle_mod):
    """eps = 0 two-body problem (e = 0.5) from pericentre to t = 2 against
    Kepler's equation: halving dt divides the position error by ~2^2 for
    the leapfrog and by ~2^6 for the seven-stage composition."""
    e2 = _kepler_errors(oracle_mod, 2, (256, 512, 1024))
    e6 = _kepler_errors(oracle_mod, 6, (32, 64, 128))
    for errs, lo, hi in ((e2, 3.6, 4.4), (e6, 48.0, 80.0)):
        r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
        assert lo < r1 < hi and lo < r2 < hi, (errs, r1, r2)
    # with fewer force evaluations (64 steps x 7 against 512) the
    # composition is far more accurate
    assert e6[1] < 1e-2 * e2[1]


def test_symplectic6_time_reversible(oracle_mod):
    m, x, v = ics.plummer(32, 4)
    x1, v1 = oracle_mod.symplectic(m, x, v, 1e-2, 1 / 64, 6, 6)
    x2, v2 = oracle_mod.symplectic(m, x1, -v1, 1e-2, 1 / 64, 6, 6)
    assert np.abs(x2 - x).max() < 1e-11 and np.abs(-v2 - v).max() < 1e-11


def test_symplectic6_order_pin_catches_a_wrong_weight(oracle_mod):
    """A weight off by one part in a thousand (the others renormalised so
    the sum stays 1) leaves a second-order error term, which the
    convergence pin above detects."""
    w = list(oracle_mod.SYMPLECTIC6_WEIGHTS)
    w[2] *= 1.001
    w[4] = w[2]
    w[3] = 1.0 - 2.0 * (w[0] + w[1] + w[2])
    errs = _kepler_errors(oracle_mod, 6, (32, 64, 128), weights=w)
    r = errs[1] / errs[2]
    assert r < 8.0, (errs, r)


def test_symplectic6_weights_are_the_best_conserving_set(oracle_mod):
    """Sec. 2.2 picks the first of the three sixth-order weight sets of its
    source table for its energy conservation, much better than with the
    other two.  The three sets are Yoshida's (1990) solutions A, B and C;
    B and C below (w1, w2, w3 as tabulated there, 15 digits) also satisfy
    the order conditions, and on an e = 0.5 Kepler orbit (dt = period / 80,
    10 orbits) the set the oracle uses keeps |dE/E| at least 5x below both,
    which is what identifies it as the paper's column."""
    others = {"B": (-2.13228522200144, 0.00426068187079180, 1.43984816797678),
              "C": (0.00152886228424922, -2.14403531630539, 1.44778256239930)}

    def max_de(ws):
        m, x, v = kepler_ic()
        E0 = oracle_mod.energy(m, x, v, 0.0)[2]
        dt = 2 * math.pi / 80
        worst = 0.0
        for _ in range(800):
            x, v = oracle_mod.symplectic(m, x, v, 0.0, dt, 1, 6, weights=ws)
            worst = max(worst, abs(oracle_mod.energy(m, x, v, 0.0)[2] / E0 - 1.0))
        return worst

    ours = max_de(None)
    for name, (w1, w2, w3) in others.items():
        w0 = 1.0 - 2.0 * (w1 + w2 + w3)
        ws = (w3, w2, w1, w0, w1, w2, w3)
        assert abs(sum(w**3 for w in ws)) < 1e-11 and abs(sum(w**5 for w in ws)) < 1e-11
        assert ours * 5.0 < max_de(ws), name
