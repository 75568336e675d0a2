"""Checks of the seeded input generators (CPU only)."""
import math

import numpy as np

from paper_0909_0879_gb300 import ics


def test_plummer_units_and_virial(oracle_mod):
    """Henon units: M = 1, centre-of-mass frame, E close to -1/4 and virial
    ratio Q = 2K/|W| close to 1 (paper Sec. 3 defines Q; Q = 1 for a
    stationary system)."""
    m, x, v = ics.plummer(4096, 1001)
    assert abs(m.sum() - 1) < 1e-14
    assert np.abs((m[:, None] * x).sum(0)).max() < 1e-14
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-14
    K, W, E = oracle_mod.energy(m, x, v, 0.0)
    assert abs(E + 0.25) < 0.02
    assert abs(2 * K / abs(W) - 1) < 0.06


def test_plummer_is_seeded():
    a = ics.plummer(100, 5)
    b = ics.plummer(100, 5)
    c = ics.plummer(100, 6)
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    assert not np.array_equal(a[1], c[1])


def test_king_profile_concentration():
    """King (1966) W0 = 7 has concentration c = log10(r_t/r_0) of about 1.53
    (the published table value); W0 = 3 has about 0.67."""
    p7 = ics.king_profile(7.0)
    assert abs(math.log10(p7["rt"]) - 1.53) < 0.02
    p3 = ics.king_profile(3.0)
    assert abs(math.log10(p3["rt"]) - 0.67) < 0.02


def test_king_sample_units(oracle_mod):
    m, x, v = ics.king(3000, 7.0, 1003)
    assert abs(m.sum() - 1) < 1e-12
    K, W, E = oracle_mod.energy(m, x, v, 0.0)
    assert abs(2 * K / abs(W) - 1) < 0.08
    assert abs(E + 0.25) < 0.03


def test_salpeter_masses():
    """Inverse-CDF sampling of dN/dm ~ m^-2.35 on [0.1, 100]: the fraction of
    stars above 1 (before normalisation) matches the analytic value."""
    m = ics.salpeter_masses(200000, 1002)
    assert abs(m.sum() - 1) < 1e-12
    assert m.max() / m.min() <= 1000.0 * (1 + 1e-12)
    e = -1.35
    frac_above_1 = (100**e - 1) / (100**e - 0.1**e)
    mm = m / m.min()  # min is ~0.1 in the raw units
    assert abs(np.mean(mm > 10.0 * (1 + 1e-3)) - frac_above_1) < 0.01


def test_uniform_sphere_virial_ratio():
    """The paper's own IC (Sec. 3): uniform sphere of radius 1 with the
    velocities rescaled to a given virial ratio; here checked against the
    continuous sphere's |W| = 3/5 (1 - sum m^2)."""
    m, x, v = ics.uniform_sphere(5000, 7, Q=0.5)
    r = np.linalg.norm(x, axis=1)
    assert r.max() <= 1.05  # radius 1 before the small centre-of-mass shift
    K = 0.5 * np.sum(m * np.sum(v * v, 1))
    assert abs(2 * K / (0.6 * (1 - np.sum(m * m))) - 0.5) < 1e-12


def test_random_subsets_and_cluster_sizes():
    idx = ics.random_active_subset(1000, 100, 3000)
    assert idx.dtype == np.int32 and len(np.unique(idx)) == 100 and np.all(np.diff(idx) > 0)
    assert np.array_equal(ics.random_active_subset(10, 10, 1), np.arange(10))
    s = ics.cluster_sizes(4096, 1004)
    assert s.min() >= 16 and s.max() <= 1024
    # log-uniform: the median is near sqrt(16 * 1024) = 128
    assert 110 < np.median(s) < 150


def test_morton_order_is_a_spatial_permutation():
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (5000, 3))
    p = ics.morton_order(x)
    assert np.array_equal(np.sort(p), np.arange(5000))
    # consecutive particles along the curve are much closer than random pairs
    d_curve = np.linalg.norm(np.diff(x[p], axis=0), axis=1).mean()
    d_rand = np.linalg.norm(np.diff(x, axis=0), axis=1).mean()
    assert d_curve < 0.2 * d_rand
    # the 8 octants come out in Z order
    pts = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [1, 1, -1],
                    [-1, -1, 1], [1, -1, 1], [-1, 1, 1], [1, 1, 1]], dtype=float)
    assert np.array_equal(ics.morton_order(pts[::-1]), np.arange(8)[::-1])
