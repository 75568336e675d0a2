"""Seeded synthetic initial conditions (inputs only).

This module generates particle sets for both the CUDA path and the FP64
oracle.  It holds none of the method's arithmetic: no pair sums, no forces,
no integrator.  Where a generator needs an energy to fix its units it uses
the analytic energy of the continuous model, never a sum over the sampled
particles.

Units are Henon units: G = M = 1 and total energy E = -1/4 for an
equilibrium model.  The paper fixes G = 1 and the total mass as the mass
unit (Sec. 3, "The NBSymple code"); the choice of E = -1/4 for the length
unit is the standard N-body convention.

Every function takes an explicit ``numpy.random.Generator`` (or an integer
seed) so that inputs are reproducible on any host.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng_for",
    "plummer",
    "king",
    "salpeter_masses",
    "uniform_sphere",
    "random_active_subset",
    "cluster_sizes",
    "morton_order",
]


def rng_for(seed) -> np.random.Generator:
    """Return a numpy Generator for an int seed or a tuple seed."""
    if isinstance(seed, np.random.Generator):
        return seed
    return np.random.default_rng(seed)


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """n unit vectors uniform on the sphere, shape (n, 3)."""
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _to_com_frame(m, x, v):
    msum = m.sum()
    x -= (m[:, None] * x).sum(axis=0) / msum
    v -= (m[:, None] * v).sum(axis=0) / msum
    return x, v


def plummer(n: int, seed, masses: np.ndarray | None = None, rmax: float = 30.0):
    """Plummer sphere in Henon units.

    Sampling after Aarseth, Henon & Wielen (1974): radius from the inverse
    cumulative mass, speed by rejection from q^2 (1 - q^2)^(7/2).  In model
    units (G = M = a = 1) the total energy is -3 pi / 64; positions are
    multiplied by 3 pi / 16 and velocities by sqrt(16 / (3 pi)) so that
    E = -1/4.  Radii beyond ``rmax`` model units are redrawn.

    Returns (m, x, v) as float64 arrays of shapes (n,), (n, 3), (n, 3),
    shifted to the centre-of-mass frame.
    """
    rng = rng_for(seed)
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
        m /= m.sum()
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        xm = rng.uniform(0.0, 1.0, todo.size)
        rr = 1.0 / np.sqrt(np.power(np.maximum(xm, 1e-300), -2.0 / 3.0) - 1.0)
        ok = rr < rmax
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    x = r[:, None] * _isotropic(rng, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.uniform(0.0, 1.0, todo.size)
        yy = rng.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * np.power(1.0 - qq * qq, 3.5)
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    speed = q * math.sqrt(2.0) * np.power(1.0 + r * r, -0.25)
    v = speed[:, None] * _isotropic(rng, n)
    x *= 3.0 * math.pi / 16.0
    v *= math.sqrt(16.0 / (3.0 * math.pi))
    x, v = _to_com_frame(m, x, v)
    return m, x, v


# ---------------------------------------------------------------- King model


def _king_rho(w):
    """King (1966) density in units of a normalisation constant, as a function
    of the dimensionless potential W >= 0 (sigma = 1)."""
    w = np.maximum(w, 0.0)
    sw = np.sqrt(w)
    from scipy.special import erf

    return np.exp(w) * erf(sw) - np.sqrt(4.0 * w / math.pi) * (1.0 + 2.0 * w / 3.0)


def king_profile(w0: float, dr: float = 1e-4):
    """Integrate the King (1966) Poisson equation W'' + 2 W'/r = -9 rho(W)/rho0.

    Radius is in units of the King radius r0 (4 pi G rho0 r0^2 = 9 sigma^2),
    sigma = 1, rho0 = rho(W0) so the central density is 1, and G = 9/(4 pi).
    RK4 in r with step ``dr`` from a series start until W crosses zero
    (the tidal radius).  Returns a dict with arrays r, W, M (enclosed mass,
    M = -r^2 W' / G) and scalars rt, Mt, Epot (model potential energy
    -G int M dM / r), all in model units.
    """
    rho0 = _king_rho(np.array([w0]))[0]
    G = 9.0 / (4.0 * math.pi)

    def rho_s(w):
        w = max(w, 0.0)
        return (math.exp(w) * math.erf(math.sqrt(w))
                - math.sqrt(4.0 * w / math.pi) * (1.0 + 2.0 * w / 3.0)) / rho0

    def rhs(r, y):
        w, dw = y
        return np.array([dw, -9.0 * rho_s(w) - 2.0 * dw / r])

    r = 1e-6
    y = np.array([w0 - 1.5 * r * r, -3.0 * r])
    rs, ws, dws = [0.0], [w0], [0.0]
    # Python-level RK4; the profile has a few hundred thousand steps at most,
    # so use an adaptive-size grid: dr grows with r (relative step <= 1e-3).
    while y[0] > 0.0:
        h = max(dr, 1e-3 * r) if r > 1.0 else dr
        k1 = rhs(r, y)
        k2 = rhs(r + 0.5 * h, y + 0.5 * h * k1)
        k3 = rhs(r + 0.5 * h, y + 0.5 * h * k2)
        k4 = rhs(r + h, y + h * k3)
        ynew = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        if ynew[0] <= 0.0:
            # linear interpolation of the zero crossing
            frac = y[0] / (y[0] - ynew[0])
            r_t = r + frac * h
            dw_t = y[1] + frac * (ynew[1] - y[1])
            rs.append(r_t)
            ws.append(0.0)
            dws.append(dw_t)
            break
        r += h
        y = ynew
        rs.append(r)
        ws.append(y[0])
        dws.append(y[1])
    r = np.array(rs)
    W = np.array(ws)
    dW = np.array(dws)
    M = -(r * r) * dW / G
    # potential energy of the continuous model, -G int M dM / r (trapezoid on
    # the integrand in M; the r -> 0 end contributes M/r -> 0)
    integrand = np.zeros_like(r)
    integrand[1:] = M[1:] / r[1:]
    Epot = -G * np.trapezoid(integrand, M)
    # the cluster's potential outside the tidal radius is -G Mt / r, so the
    # potential inside is Phi = -W + Phi(rt); Epot above is already the full
    # self-energy because it integrates the pair interaction directly.
    return {"r": r, "W": W, "M": M, "rt": r[-1], "Mt": M[-1], "Epot": Epot, "G": G}


_KING_CACHE: dict = {}


def king(n: int, w0: float, seed):
    """King (1966) model with central potential W0, equal masses, Henon units.

    Radii are drawn from the tabulated enclosed mass M(r); speeds at radius r
    by rejection from v^2 (exp(W(r) - v^2/2) - 1) on [0, sqrt(2 W(r))]
    (the lowered-isothermal distribution with sigma = 1); directions
    isotropic.  Units: the continuous model is an equilibrium, so its total
    energy is Epot/2 (virial theorem); masses are scaled so M = 1 and the
    velocity and length scales V^2 = -4 E / M, L = G M / V^2 make G = 1 and
    E = -1/4.  The sampled set's own energy differs from -1/4 by sampling
    noise of order N^(-1/2).
    """
    rng = rng_for(seed)
    key = float(w0)
    if key not in _KING_CACHE:
        _KING_CACHE[key] = king_profile(w0)
    prof = _KING_CACHE[key]
    r_tab, W_tab, M_tab = prof["r"], prof["W"], prof["M"]
    Mt = prof["Mt"]
    u = rng.uniform(0.0, 1.0, n) * Mt
    r = np.interp(u, M_tab, r_tab)
    W = np.maximum(np.interp(r, r_tab, W_tab), 0.0)
    vmax = np.sqrt(2.0 * W)
    # envelope: maximum of g(v) on a 64-point grid, times a safety factor
    grid = np.linspace(0.0, 1.0, 65)[1:]
    gmax = np.zeros(n)
    for s in grid:
        vv = s * vmax
        gmax = np.maximum(gmax, vv * vv * (np.exp(W - 0.5 * vv * vv) - 1.0))
    gmax *= 1.1
    speed = np.zeros(n)
    todo = np.nonzero(vmax > 0.0)[0]
    while todo.size:
        vv = rng.uniform(0.0, 1.0, todo.size) * vmax[todo]
        yy = rng.uniform(0.0, 1.0, todo.size) * gmax[todo]
        g = vv * vv * (np.exp(W[todo] - 0.5 * vv * vv) - 1.0)
        ok = yy < g
        speed[todo[ok]] = vv[ok]
        todo = todo[~ok]
    x = r[:, None] * _isotropic(rng, n)
    v = speed[:, None] * _isotropic(rng, n)
    G = prof["G"]
    E = 0.5 * prof["Epot"]
    V2 = -4.0 * E / Mt
    L = G * Mt / V2
    x /= L
    v /= math.sqrt(V2)
    m = np.full(n, 1.0 / n)
    x, v = _to_com_frame(m, x, v)
    return m, x, v


# ------------------------------------------------------------- mass spectra


def salpeter_masses(n: int, seed, lo: float = 0.1, hi: float = 100.0, alpha: float = 2.35):
    """Masses from dN/dm ~ m^-alpha on [lo, hi] by the inverse CDF, then
    normalised to a total of 1."""
    rng = rng_for(seed)
    u = rng.uniform(0.0, 1.0, n)
    e = 1.0 - alpha
    m = np.power(lo**e + u * (hi**e - lo**e), 1.0 / e)
    return m / m.sum()


def uniform_sphere(n: int, seed, Q: float = 1.0, masses: np.ndarray | None = None):
    """The paper's own test system (Sec. 3): positions uniform in a sphere of
    radius 1, velocities uniform in direction and in magnitude on [0, 1],
    then rescaled to the virial ratio Q = 2K/|W|.  M = 1, G = 1.

    |W| is taken from the continuous uniform sphere, 3/5 (1 - sum m_i^2)
    (the sum removes the self-energy a discrete set does not have), so no
    pair sum is evaluated here.
    """
    rng = rng_for(seed)
    m = np.full(n, 1.0 / n) if masses is None else np.asarray(masses, float) / np.sum(masses)
    r = np.cbrt(rng.uniform(0.0, 1.0, n))
    x = r[:, None] * _isotropic(rng, n)
    s = rng.uniform(0.0, 1.0, n)
    v = s[:, None] * _isotropic(rng, n)
    x, v = _to_com_frame(m, x, v)
    w_abs = 0.6 * (1.0 - np.sum(m * m))
    kin = 0.5 * np.sum(m * np.sum(v * v, axis=1))
    if kin > 0.0:
        v *= math.sqrt(Q * w_abs / (2.0 * kin))
    return m, x, v


# -------------------------------------------------------------- index sets


def random_active_subset(n: int, n_act: int, seed) -> np.ndarray:
    """n_act distinct indices of [0, n), drawn without replacement, sorted
    ascending, int32."""
    rng = rng_for(seed)
    if n_act >= n:
        return np.arange(n, dtype=np.int32)
    idx = rng.choice(n, size=n_act, replace=False)
    return np.sort(idx).astype(np.int32)


def cluster_sizes(n_clusters: int, seed, lo: int = 16, hi: int = 1024) -> np.ndarray:
    """Cluster sizes round(exp(U(ln lo, ln hi))), int64."""
    rng = rng_for(seed)
    s = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n_clusters)))
    return np.clip(s, lo, hi).astype(np.int64)


def morton_order(x: np.ndarray, bits: int = 21) -> np.ndarray:
    """Permutation that lists particles along a Morton (Z-order) curve of
    their positions: coordinates are quantised to ``bits`` bits over the
    bounding cube and interleaved into one integer key.  Spatially close
    particles get close indices (a data-layout choice; it changes no
    value)."""
    x = np.asarray(x, dtype=np.float64)
    lo = x.min(axis=0)
    span = float((x.max(axis=0) - lo).max()) or 1.0
    q = np.minimum(((x - lo) / span * (2**bits - 1)).astype(np.uint64), np.uint64(2**bits - 1))

    def spread(v):
        v = v & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v

    key = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1)) | (spread(q[:, 2]) << np.uint64(2))
    return np.argsort(key, kind="stable")
