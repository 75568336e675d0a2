"""Pins for the oracle's external Galactic field (Allen & Santillan 1991,
the field the paper's Sec. 2.1 adds to the pair forces) and for the
symplectic and Hermite integrators with it (CPU only)."""
import math

import numpy as np

R0 = 8.5  # kpc


def test_circular_speed_at_the_sun(oracle_mod):
    """Allen & Santillan calibrate the model to a circular speed of 220 km/s
    (22 units of 10 km/s) at R0 = 8.5 kpc."""
    a, _ = oracle_mod.ext_field([[R0, 0.0, 0.0]])
    assert abs(a[0, 1]) == 0.0 and abs(a[0, 2]) == 0.0
    vc = math.sqrt(-a[0, 0] * R0)
    assert abs(vc - 22.0) < 0.01, vc


def test_acceleration_is_minus_gradient_of_potential(oracle_mod):
    """Central differences of the potential at points in and off the disk
    plane, near the axis, near the centre and beyond the halo's cut."""
    rng = np.random.default_rng(1)
    pts = np.concatenate([
        rng.normal(0.0, 6.0, (12, 3)),
        [[R0, 0.0, 0.0], [0.05, 0.02, 0.3], [0.0, 0.0, 2.0], [3.0, -1.0, 0.01],
         [80.0, 40.0, 30.0], [150.0, -20.0, 60.0]]])
    a, _ = oracle_mod.ext_field(pts)
    for p, ap in zip(pts, a):
        h = 1e-5 * max(1.0, np.linalg.norm(p))
        g = np.zeros(3)
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            g[c] = (oracle_mod.ext_field([p + e])[1][0] - oracle_mod.ext_field([p - e])[1][0]) / (2 * h)
        assert np.linalg.norm(ap + g) <= 1e-7 * np.linalg.norm(ap), (p, ap, -g)


def test_disk_with_zero_scale_length_is_a_plummer_sphere(oracle_mod):
    """Miyamoto-Nagai with a = 0 reduces to a Plummer sphere of scale b."""
    pts = np.random.default_rng(2).normal(0.0, 3.0, (20, 3))
    only_disk = {"m_bulge": 0.0, "m_halo": 0.0, "a_disk": 0.0, "b_disk": 0.7}
    only_bulge = {"m_disk": 0.0, "m_halo": 0.0, "m_bulge": 3690.0, "b_bulge": 0.7}
    a1, p1 = oracle_mod.ext_field(pts, only_disk)
    a2, p2 = oracle_mod.ext_field(pts, only_bulge)
    assert np.allclose(a1, a2, rtol=1e-13, atol=0) and np.allclose(p1, p2, rtol=1e-13, atol=0)


def test_halo_potential_continuous_and_keplerian_beyond_cut(oracle_mod):
    """The halo's closed-form potential inside the cut meets the Keplerian
    -G M(r_cut) / r outside; far away the whole field is that of a point
    of mass M_b + M_d + M_h(r_cut)."""
    halo = {"m_bulge": 0.0, "m_disk": 0.0}
    rc = 100.0
    _, pin = oracle_mod.ext_field([[rc * (1 - 1e-9), 0, 0]], halo)
    _, pout = oracle_mod.ext_field([[rc * (1 + 1e-9), 0, 0]], halo)
    q = rc / 12.0
    mcut = 4615.0 * q**2.02 / (1 + q**1.02)
    assert abs(pout[0] + mcut / (rc * (1 + 1e-9))) < 1e-12 * abs(pout[0])
    assert abs(pin[0] - pout[0]) < 1e-6 * abs(pout[0])
    r = 1e7
    _, pfar = oracle_mod.ext_field([[0, 0, r]])
    assert abs(pfar[0] * r + (606.0 + 3690.0 + mcut)) < 1e-5 * (606.0 + 3690.0 + mcut)


def test_circular_orbit_closed_form(oracle_mod):
    """A test particle on the circular orbit at R0 in the plane moves
    uniformly, x(t) = R0 (cos wt, sin wt, 0) with w = v_c / R0: the sixth-
    order composition follows it over a quarter period, and halving dt
    divides the error by ~2^6."""
    a, _ = oracle_mod.ext_field([[R0, 0.0, 0.0]])
    vc = math.sqrt(-a[0, 0] * R0)
    w = vc / R0
    t_end = 0.25 * 2 * math.pi / w
    m = np.array([1e-12])
    errs = []
    for k in (16, 32):
        x, v = oracle_mod.symplectic(m, [[R0, 0.0, 0.0]], [[0.0, vc, 0.0]], 0.0, t_end / k, k, 6,
                                     ext={})
        exact = R0 * np.array([math.cos(w * t_end), math.sin(w * t_end), 0.0])
        errs.append(np.linalg.norm(x[0] - exact))
    assert errs[1] < 1e-6 * R0
    assert 40.0 < errs[0] / errs[1] < 90.0, errs


def test_energy_conserved_on_an_eccentric_orbit(oracle_mod):
    """A bound, inclined, eccentric orbit through bulge, disk and halo: the
    energy 1/2 v^2 + Phi of the sixth-order run stays within 1e-9 over two
    units of time (about one orbit) at dt = 1/512."""
    m = np.array([1e-12])
    x = np.array([[6.0, 0.0, 1.0]])
    v = np.array([[0.0, 15.0, 8.0]])
    E0 = 0.5 * np.sum(v**2) + oracle_mod.ext_field(x)[1][0]
    worst = 0.0
    for _ in range(8):
        x, v = oracle_mod.symplectic(m, x, v, 0.0, 1.0 / 512, 128, 6, ext={})
        E = 0.5 * np.sum(v**2) + oracle_mod.ext_field(x)[1][0]
        worst = max(worst, abs(E / E0 - 1.0))
    assert worst < 1e-9, worst


def test_field_jerk_is_time_derivative_of_acceleration(oracle_mod):
    """The jerk d a(x + v t)/dt at t = 0 against central differences along
    the straight line, at points in and off the plane, near the axis, near
    the centre and beyond the halo cut, with random velocities."""
    rng = np.random.default_rng(4)
    pts = np.concatenate([
        rng.normal(0.0, 6.0, (12, 3)),
        [[R0, 0.0, 0.0], [0.05, 0.02, 0.3], [0.0, 0.0, 2.0], [3.0, -1.0, 0.01],
         [80.0, 40.0, 30.0], [150.0, -20.0, 60.0]]])
    vel = rng.normal(0.0, 15.0, pts.shape)
    _, _, jk = oracle_mod.ext_field(pts, v=vel)
    for p, u, jp in zip(pts, vel, jk):
        h = 1e-6 * max(1.0, np.linalg.norm(p)) / max(1.0, np.linalg.norm(u))
        ap = oracle_mod.ext_field([p + u * h])[0][0]
        am = oracle_mod.ext_field([p - u * h])[0][0]
        fd = (ap - am) / (2 * h)
        assert np.linalg.norm(jp - fd) <= 1e-6 * np.linalg.norm(fd), (p, jp, fd)


def test_hermite_with_field_circular_orbit(oracle_mod):
    """A test particle on the circular orbit at R0, Hermite-4 with shared
    steps and the field's acceleration and jerk: fourth-order convergence
    towards the uniform circular motion over a fifth of a period."""
    a, _ = oracle_mod.ext_field([[R0, 0.0, 0.0]])
    vc = math.sqrt(-a[0, 0] * R0)
    w = vc / R0
    m = np.array([1e-12])
    errs = []
    t_end = 0.5  # a fifth of the 2.43-unit period
    for lev in (6, 7, 8):
        x, v, _, _ = oracle_mod.hermite_shared(m, [[R0, 0.0, 0.0]], [[0.0, vc, 0.0]], 0.0, lev,
                                               int(t_end * 2**lev), ext={})
        exact = R0 * np.array([math.cos(w * t_end), math.sin(w * t_end), 0.0])
        errs.append(np.linalg.norm(x[0] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12.0 < r1 < 20.0 and 12.0 < r2 < 20.0, errs
    assert errs[2] < 1e-8 * R0


def test_field_centre_is_a_translation(oracle_mod):
    """The field about a centre c at x equals the field about the origin at
    x - c (acceleration, jerk and potential)."""
    rng = np.random.default_rng(5)
    pts = rng.normal(0.0, 5.0, (10, 3))
    vel = rng.normal(0.0, 10.0, (10, 3))
    c = np.array([1.5, -2.0, 0.7])
    a1, p1, j1 = oracle_mod.ext_field(pts, {"center": tuple(c)}, v=vel)
    a2, p2, j2 = oracle_mod.ext_field(pts - c, v=vel)
    assert np.allclose(a1, a2, rtol=1e-14, atol=0)
    assert np.allclose(j1, j2, rtol=1e-14, atol=1e-14 * np.abs(j2).max())
    assert np.allclose(p1, p2, rtol=1e-14, atol=0)
