"""Pins for the oracle's force, jerk and energy (CPU only).

Each test checks the oracle against something other than its own formula:
high-precision arithmetic on a differently written expression, conservation
laws, closed forms, finite differences, or an identity that ties the force
to the energy.
"""
import math

import numpy as np
import pytest

from paper_0909_0879_gb300 import ics


def _rand_system(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.1, 1.0, n)
    x = rng.normal(0.0, spread, (n, 3))
    v = rng.normal(0.0, 1.0, (n, 3))
    return m, x, v


@pytest.mark.parametrize("n,eps", [(2, 0.0), (3, 0.1), (5, 0.01), (8, 0.3)])
def test_force_jerk_vs_50_digit_gradient(oracle_mod, n, eps):
    """Acceleration as minus the gradient of the softened potential and jerk
    as the time derivative of the acceleration along the flow, both by
    50-digit numerical differentiation (mpmath), eq. (1) with Plummer
    softening."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    m, x, v = _rand_system(n, 100 + n)
    acc, jerk = oracle_mod.force_jerk(m, x, v, eps)
    M = [mp.mpf(float(q)) for q in m]
    X = [[mp.mpf(float(q)) for q in row] for row in x]
    V = [[mp.mpf(float(q)) for q in row] for row in v]
    e2 = mp.mpf(float(eps)) ** 2

    def phi_i(i, xi):
        # potential per unit mass at xi from every j != i
        s = mp.mpf(0)
        for j in range(n):
            if j == i:
                continue
            r2 = sum((X[j][c] - xi[c]) ** 2 for c in range(3))
            s -= M[j] / mp.sqrt(r2 + e2)
        return s

    def acc_at(i, t):
        # acceleration on i with every particle moved along x + v t,
        # written as minus the gradient of the potential in closed form
        xi = [X[i][c] + V[i][c] * t for c in range(3)]
        out = [mp.mpf(0)] * 3
        for j in range(n):
            if j == i:
                continue
            xj = [X[j][c] + V[j][c] * t for c in range(3)]
            r2 = sum((xj[c] - xi[c]) ** 2 for c in range(3)) + e2
            for c in range(3):
                out[c] += M[j] * (xj[c] - xi[c]) / r2 ** mp.mpf(1.5)
        return out

    for i in range(n):
        for c in range(3):
            def f(h, i=i, c=c):
                xi = list(X[i])
                xi[c] = xi[c] + h
                return phi_i(i, xi)

            a_ref = -mp.diff(f, 0)
            assert abs(float(a_ref) - acc[i, c]) <= 1e-12 * (1 + abs(float(a_ref)))
            j_ref = mp.diff(lambda t, i=i, c=c: acc_at(i, t)[c], 0)
            assert abs(float(j_ref) - jerk[i, c]) <= 1e-12 * (1 + abs(float(j_ref)))


def test_two_body_closed_form(oracle_mod):
    """Two bodies: a_1 = G m_2 d/(d^2+eps^2)^(3/2) and the jerk closed form,
    worked by hand for d = (3, 4, 0), eps = 0 and w = (0, 1, 0)."""
    m = np.array([2.0, 5.0])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    acc, jerk = oracle_mod.force_jerk(m, x, v, 0.0, G=1.0)
    # |d| = 5: a_1 = 5 * (3,4,0)/125 = (0.12, 0.16, 0)
    np.testing.assert_allclose(acc[0], [0.12, 0.16, 0.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(acc[1], [-0.048, -0.064, 0.0], rtol=0, atol=1e-15)
    # jerk_1 = m2 [w/125 - 3 (d.w) d / 5^5] with d.w = 4:
    #        = 5 [(0, 0.008, 0) - 12 (3,4,0)/3125] = (-0.0576, -0.0368, 0)
    np.testing.assert_allclose(jerk[0], [-0.0576, -0.0368, 0.0], rtol=0, atol=1e-15)
    # Newton's third law on the pair
    np.testing.assert_allclose(m[0] * jerk[0], -m[1] * jerk[1], atol=1e-15)
    # softened: eps = 5 doubles s^2 -> a scaled by 2^-1.5
    acc_s, _ = oracle_mod.force_jerk(m, x, v, 5.0, G=2.0)
    np.testing.assert_allclose(acc_s[0], 2.0 * np.array([0.12, 0.16, 0.0]) / 2**1.5, atol=1e-15)


@pytest.mark.parametrize("eps", [0.0, 1e-3, 0.05])
def test_newton_third_law_and_torque(oracle_mod, eps):
    """sum m a = 0, sum m jerk = 0 and sum m x cross a = 0 (pair forces are
    equal, opposite and central)."""
    m, x, v = ics.plummer(300, 7)
    acc, jerk = oracle_mod.force_jerk(m, x, v, eps)
    scale_a = np.sum(m[:, None] * np.abs(acc))
    scale_j = np.sum(m[:, None] * np.abs(jerk))
    assert np.all(np.abs((m[:, None] * acc).sum(0)) < 1e-13 * scale_a)
    assert np.all(np.abs((m[:, None] * jerk).sum(0)) < 1e-13 * scale_j)
    torque = (m[:, None] * np.cross(x, acc)).sum(0)
    assert np.all(np.abs(torque) < 1e-13 * np.sum(m * np.linalg.norm(x, axis=1) * np.linalg.norm(acc, axis=1)))


def test_virial_identity_ties_force_to_energy(oracle_mod):
    """With eps = 0 the pair potential is homogeneous of degree -1, so
    sum_i m_i x_i . a_i = W exactly (Euler's theorem); with eps > 0,
    sum_i m_i x_i . a_i = -sum_{i<j} m_i m_j r^2 / s^3 = W + eps^2 sum m_i m_j / s^3."""
    m, x, v = ics.plummer(400, 11)
    acc, _ = oracle_mod.force_jerk(m, x, v, 0.0)
    _, W, _ = oracle_mod.energy(m, x, v, 0.0)
    vir = np.sum(m[:, None] * x * acc)
    assert abs(vir - W) < 1e-12 * abs(W)
    eps = 0.05
    acc, _ = oracle_mod.force_jerk(m, x, v, eps)
    _, W, _ = oracle_mod.energy(m, x, v, eps)
    d = x[None, :, :] - x[:, None, :]
    s2 = np.sum(d * d, axis=2) + eps * eps
    iu = np.triu_indices(len(m), 1)
    extra = np.sum((m[:, None] * m[None, :])[iu] * eps * eps / s2[iu] ** 1.5)
    vir = np.sum(m[:, None] * x * acc)
    assert abs(vir - (W + extra)) < 1e-12 * abs(W)


def test_force_is_minus_energy_gradient(oracle_mod):
    """m_i a_i = -dW/dx_i, checked by central differences of the oracle's own
    energy (a different routine) in FP64."""
    m, x, v = _rand_system(12, 5)
    eps = 0.02
    acc, _ = oracle_mod.force_jerk(m, x, v, eps)
    h = 1e-5
    for i in range(12):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            dW = (oracle_mod.energy(m, xp, v, eps)[1] - oracle_mod.energy(m, xm, v, eps)[1]) / (2 * h)
            assert abs(-dW - m[i] * acc[i, c]) < 1e-7 * (1 + abs(dW))


def test_jerk_is_flow_derivative_of_acc(oracle_mod):
    """jerk = d/dt a(x + v t) at t = 0, central differences with every
    particle advanced (O(h^2) accurate)."""
    m, x, v = ics.plummer(200, 3)
    eps = 1e-2
    _, jerk = oracle_mod.force_jerk(m, x, v, eps)
    h = 1e-5
    ap, _ = oracle_mod.force_jerk(m, x + v * h, v, eps)
    am, _ = oracle_mod.force_jerk(m, x - v * h, v, eps)
    fd = (ap - am) / (2 * h)
    err = np.abs(fd - jerk).max() / np.abs(jerk).max()
    assert err < 1e-6


def test_idx_subset_and_thread_independence(oracle_mod):
    """The i-subset path returns the same rows as the full evaluation, and
    the result does not depend on the OpenMP thread count (fixed j order)."""
    m, x, v = ics.plummer(500, 9)
    a_all, j_all = oracle_mod.force_jerk(m, x, v, 1e-3)
    idx = np.array([499, 0, 17, 250, 17])
    a_s, j_s = oracle_mod.force_jerk(m, x, v, 1e-3, idx=idx)
    assert np.array_equal(a_s, a_all[idx]) and np.array_equal(j_s, j_all[idx])
    nt = oracle_mod.max_threads()
    oracle_mod.set_threads(1)
    try:
        a_1, j_1 = oracle_mod.force_jerk(m, x, v, 1e-3)
    finally:
        oracle_mod.set_threads(nt)
    assert np.array_equal(a_1, a_all) and np.array_equal(j_1, j_all)


def test_energy_two_body_closed_form(oracle_mod):
    m = np.array([2.0, 5.0])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 2.0]])
    K, W, E = oracle_mod.energy(m, x, v, 0.0)
    assert K == 0.5 * 2.0 * 1.0 + 0.5 * 5.0 * 8.0
    assert abs(W - (-10.0 / 5.0)) < 1e-15
    K, W, E = oracle_mod.energy(m, x, v, 5.0, G=3.0)
    assert abs(W - (-3.0 * 10.0 / math.sqrt(50.0))) < 1e-14


def test_plummer_mean_field(oracle_mod):
    """Statistical pin: in Henon units a Plummer sphere's mean field is
    a(r) = -r / (r^2 + b^2)^(3/2) with b = 3 pi / 16.  Averaged over shells,
    the N-body acceleration follows it to within sampling noise."""
    n = 4000
    m, x, v = ics.plummer(n, 21)
    acc, _ = oracle_mod.force_jerk(m, x, v, 1e-3)
    b = 3 * math.pi / 16
    r = np.linalg.norm(x, axis=1)
    a_rad = -np.sum(acc * x, axis=1) / r
    analytic = r / (r * r + b * b) ** 1.5
    sel = (r > 0.2) & (r < 2.0)
    ratio = np.mean(a_rad[sel]) / np.mean(analytic[sel])
    assert abs(ratio - 1.0) < 0.05


def test_interaction_count_matches_table1(oracle_mod):
    """The paper's cost model (Sec. 2, Table 1): n_f = 30 N (N-1)/2 flops per
    force evaluation.  The golden file holds the printed table; our pair
    counter N(N-1)/2 reproduces its n_f column to the two printed digits."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "table1_cost_model.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    from paper_0909_0879_gb300.metrics import pair_count

    for name, n, nf, tcpu in rows:
        n, nf = float(n), float(nf)
        mine = 30.0 * pair_count(n)
        assert abs(mine - nf) / nf < 0.01, (name, mine, nf)


def test_condition_sums(oracle_mod):
    """sum_j |f_ij| >= |a_i| (triangle inequality), with equality when every
    pair term points the same way (all other bodies on one ray from i), and
    it is |a| for two bodies."""
    m, x, v = ics.plummer(300, 17)
    acc, jerk = oracle_mod.force_jerk(m, x, v, 1e-3)
    aabs, jabs = oracle_mod.force_jerk_abs(m, x, v, 1e-3)
    assert np.all(aabs >= np.linalg.norm(acc, axis=1) * (1 - 1e-14))
    assert np.all(jabs >= np.linalg.norm(jerk, axis=1) * (1 - 1e-14))
    xr = np.zeros((5, 3))
    xr[:, 0] = [0.0, 1.0, 2.5, 3.0, 7.0]
    vr = np.zeros((5, 3))
    vr[:, 0] = [0.0, 0.1, 0.3, -0.2, 0.5]
    mr = np.array([1.0, 0.5, 2.0, 0.25, 3.0])
    a, jk = oracle_mod.force_jerk(mr, xr, vr, 0.0)
    aa, ja = oracle_mod.force_jerk_abs(mr, xr, vr, 0.0)
    assert abs(aa[0] - np.linalg.norm(a[0])) < 1e-14 * aa[0]
    # on a line with radial velocities every jerk term is radial too, but the
    # signs differ; the sum of magnitudes bounds it
    assert ja[0] >= np.linalg.norm(jk[0])
    a2, j2 = oracle_mod.force_jerk(mr[:2], xr[:2], vr[:2] + [[0, 0.3, 0]] * 2, 0.1)
    aa2, ja2 = oracle_mod.force_jerk_abs(mr[:2], xr[:2], vr[:2] + [[0, 0.3, 0]] * 2, 0.1)
    assert np.allclose(aa2, np.linalg.norm(a2, axis=1), rtol=1e-14)
    assert np.allclose(ja2, np.linalg.norm(j2, axis=1), rtol=1e-14)
