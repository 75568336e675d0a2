"""Python access to the FP64 CPU oracle (``nbody_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check
in ``__graft_entry__.py`` and by the CPU-baseline leg of ``bench.py``.  The
product path never imports it.  It shares nothing with the CUDA library but
the seeded input generators that produce its inputs.

``build()`` compiles the C file with gcc (``-O3 -fopenmp -ffp-contract=off``,
no machine-specific flags) into ``oracle/_build/liboracle.so``; ``lib()``
builds on first use when the shared object is missing or older than the
source.  ``compile_to(src, out)`` builds any copy of the source the same way.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nbody_oracle.c")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "liboracle.so")
# A test that checks that the pins catch planted mistakes points this at a
# deliberately broken copy of the oracle built in a temporary directory.
_SO_OVERRIDE = os.environ.get("NBODY_ORACLE_SO")
TICKS_LOG2 = 20

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if _SO_OVERRIDE:
        return _SO_OVERRIDE
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        tmp = SO + f".tmp{os.getpid()}"
        compile_to(SRC, tmp)
        os.replace(tmp, SO)
    return SO


def compile_to(src: str, out: str) -> str:
    cmd = ["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c11", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i64, i32, vp = C.c_double, C.c_int64, C.c_int32, C.c_void_p
            L.orc_max_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_force_jerk.argtypes = [i64, vp, vp, vp, d, d, i64, vp, vp, vp]
            L.orc_force_jerk_abs.argtypes = [i64, vp, vp, vp, d, d, i64, vp, vp, vp]
            L.orc_energy.argtypes = [i64, vp, vp, vp, d, d, vp, vp]
            L.orc_predict.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
            L.orc_aarseth_dt.argtypes = [vp, vp, vp, vp, d]
            L.orc_aarseth_dt.restype = d
            L.orc_level_from_dt.argtypes = [d, C.c_int, C.c_int, vp]
            L.orc_level_from_dt.restype = C.c_int
            L.orc_next_level.argtypes = [C.c_int, C.c_int, i64, C.c_int]
            L.orc_next_level.restype = C.c_int
            L.orc_hermite_init.argtypes = [i64, vp, vp, vp, d, d, d, C.c_int, C.c_int,
                                           vp, vp, vp, vp]
            L.orc_block_step.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, d, d, d,
                                         C.c_int, C.c_int, C.c_int, i64, i64, vp,
                                         vp, vp, vp]
            L.orc_block_step.restype = i64
            L.orc_hermite_shared.argtypes = [i64, vp, vp, vp, vp, vp, d, d, C.c_int, i64]
            L.orc_acc.argtypes = [i64, vp, vp, d, d, vp]
            L.orc_leapfrog.argtypes = [i64, vp, vp, vp, d, d, d, i64]
            L.orc_acc_vjp.argtypes = [i64, vp, vp, d, d, vp, vp, vp]
            L.orc_leapfrog_loss_grad.argtypes = [i64, vp, vp, vp, vp, d, d, d, i64,
                                                 vp, vp, vp]
            L.orc_leapfrog_loss_grad.restype = d
            L.orc_leapfrog_adjoint_path.argtypes = [i64, vp, vp, d, d, d, i64, vp, vp, vp]
            L.orc_ext.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            L.orc_hermite_init_ext.argtypes = [i64, vp, vp, vp, d, d, d, C.c_int, C.c_int,
                                               vp, vp, vp, vp, vp]
            L.orc_block_step_ext.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, d, d, d,
                                             C.c_int, C.c_int, C.c_int, i64, i64, vp, vp,
                                             vp, vp, vp]
            L.orc_block_step_ext.restype = i64
            _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def max_threads() -> int:
    return lib().orc_max_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def force_jerk(m, x, v, eps, G=1.0, idx=None):
    """Acceleration and jerk on particles ``idx`` (all when None) from all
    others.  Returns (acc, jerk) of shape (n_i, 3)."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    if idx is None:
        n_i, ip = n, None
    else:
        ip = np.ascontiguousarray(idx, dtype=np.int64)
        n_i = ip.shape[0]
    acc = np.zeros((n_i, 3))
    jerk = np.zeros((n_i, 3))
    lib().orc_force_jerk(n, _p(m), _p(x), _p(v), float(G), float(eps), n_i, _p(ip),
                         _p(acc), _p(jerk))
    return acc, jerk


def force_jerk_abs(m, x, v, eps, G=1.0, idx=None):
    """Sums of the magnitudes of the pair terms of the acceleration and the
    jerk on particles ``idx`` (the condition of each sum).  Returns two
    arrays of shape (n_i,)."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    if idx is None:
        n_i, ip = n, None
    else:
        ip = np.ascontiguousarray(idx, dtype=np.int64)
        n_i = ip.shape[0]
    aabs = np.zeros(n_i)
    jabs = np.zeros(n_i)
    lib().orc_force_jerk_abs(n, _p(m), _p(x), _p(v), float(G), float(eps), n_i, _p(ip),
                             _p(aabs), _p(jabs))
    return aabs, jabs


def acc(m, x, eps, G=1.0):
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    out = np.zeros((n, 3))
    lib().orc_acc(n, _p(m), _p(x), float(G), float(eps), _p(out))
    return out


def energy(m, x, v, eps, G=1.0):
    """Returns (K, W, E) with the softened pair potential."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    k = np.zeros(1)
    w = np.zeros(1)
    lib().orc_energy(n, _p(m), _p(x), _p(v), float(G), float(eps), _p(k), _p(w))
    return float(k[0]), float(w[0]), float(k[0] + w[0])


def predict(x, v, a, jk, dt):
    x, v, a, jk = (_f64(q).reshape(-1, 3) for q in (x, v, a, jk))
    n = x.shape[0]
    dt = np.broadcast_to(np.asarray(dt, np.float64), (n,)).copy()
    xp = np.zeros_like(x)
    vp = np.zeros_like(v)
    lib().orc_predict(n, _p(x), _p(v), _p(a), _p(jk), _p(dt), _p(xp), _p(vp))
    return xp, vp


def aarseth_dt(a, jk, a2, a3, eta):
    a, jk, a2, a3 = (_f64(q) for q in (a, jk, a2, a3))
    return lib().orc_aarseth_dt(_p(a), _p(jk), _p(a2), _p(a3), float(eta))


def level_from_dt(dt, lev_min=3, lev_max=20):
    cl = np.zeros(1, dtype=np.int32)
    lev = lib().orc_level_from_dt(float(dt), int(lev_min), int(lev_max), _p(cl))
    return lev, bool(cl[0])


def next_level(lev_old, lev_want, t_new, lev_min=3):
    return lib().orc_next_level(int(lev_old), int(lev_want), int(t_new), int(lev_min))


class HermiteState:
    """FP64 state of a Hermite-4 integration in the oracle (arrays owned by
    Python).  ``block_levels`` selects the Aarseth block-step scheme; with it
    off every particle keeps its level (shared fixed dt = 2^-lev).  ``ext``
    (a dict of external-field parameters, {} for Allen & Santillan's) adds
    the field's acceleration and jerk to the pair sums (Sec. 2.1)."""

    def __init__(self, m, x, v, eps, G=1.0, eta=0.01, eta_start=0.01, lev_min=3,
                 lev_max=20, block_levels=True, shared_lev=None, ext=None):
        self.m = _f64(m).copy()
        n = self.n = self.m.shape[0]
        self.x = _f64(x, (n, 3)).copy()
        self.v = _f64(v, (n, 3)).copy()
        self.a = np.zeros((n, 3))
        self.jk = np.zeros((n, 3))
        self.lev = np.zeros(n, dtype=np.int32)
        self.t = np.zeros(n, dtype=np.int64)
        self.G, self.eps, self.eta = float(G), float(eps), float(eta)
        self.lev_min, self.lev_max = int(lev_min), int(lev_max)
        self.block_levels = bool(block_levels)
        self.n_clamped = np.zeros(1, dtype=np.int64)
        self._ext = None if ext is None else _ext_params(ext)
        lib().orc_hermite_init_ext(n, _p(self.m), _p(self.x), _p(self.v), self.G, self.eps,
                                   float(eta_start), self.lev_min, self.lev_max,
                                   _p(self._ext), _p(self.a), _p(self.jk), _p(self.lev),
                                   _p(self.t))
        if shared_lev is not None:
            self.lev[:] = int(shared_lev)
        self._act = np.zeros(n, dtype=np.int64)

    def step(self, replay=None):
        """One block step; ``replay`` = (t_next_tick, active indices) follows a
        given schedule.  Returns (t_next_tick, active indices)."""
        tn = np.zeros(1, dtype=np.int64)
        if replay is None:
            rt, rn, ra = 0, -1, None
        else:
            rt = int(replay[0])
            ra = np.ascontiguousarray(replay[1], dtype=np.int64)
            rn = ra.shape[0]
        n_act = lib().orc_block_step_ext(
            self.n, _p(self.m), _p(self.x), _p(self.v), _p(self.a), _p(self.jk),
            _p(self.t), _p(self.lev), self.G, self.eps, self.eta, self.lev_min,
            self.lev_max, int(self.block_levels), rt, rn, _p(ra), _p(self._ext), _p(tn),
            _p(self._act), _p(self.n_clamped))
        return int(tn[0]), self._act[:n_act].copy()

    def time(self) -> float:
        return float(self.t.max()) * 2.0 ** (-TICKS_LOG2)

    def energy(self):
        """(K, W, E); with an external field W includes sum m Phi_ext."""
        K, W, E = energy(self.m, self.x, self.v, self.eps, self.G)
        if self._ext is not None:
            phi = np.zeros(self.n)
            lib().orc_ext(self.n, _p(self.x), None, _p(self._ext), None, None, _p(phi))
            W_ext = float(np.sum(self.m * phi))
            W, E = W + W_ext, E + W_ext
        return K, W, E


def hermite_shared(m, x, v, eps, lev, nsteps, G=1.0, ext=None):
    """Shared fixed dt = 2^-lev; returns (x, v, a, jerk) after nsteps."""
    st = HermiteState(m, x, v, eps, G=G, block_levels=False, shared_lev=lev, ext=ext)
    for _ in range(nsteps):
        st.step()
    return st.x, st.v, st.a, st.jk


def leapfrog(m, x, v, eps, dt, nsteps, G=1.0):
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3)).copy()
    v = _f64(v, (n, 3)).copy()
    lib().orc_leapfrog(n, _p(m), _p(x), _p(v), float(G), float(eps), float(dt), int(nsteps))
    return x, v


# Sec. 2.2: the sixth-order scheme is a symmetric composition of seven
# leapfrog steps of lengths w_k dt.  Weights: Yoshida (1990, Phys. Lett. A
# 150, 262), solution A, which is the first of the three sixth-order sets
# tabulated by Kinoshita, Yoshida & Nakai (1991, Table 1), the set the paper
# takes for its energy conservation.
SYMPLECTIC6_W1 = -1.17767998417887100695
SYMPLECTIC6_W2 = 0.235573213359358133684
SYMPLECTIC6_W3 = 0.784513610477557263820
SYMPLECTIC6_W0 = 1.0 - 2.0 * (SYMPLECTIC6_W1 + SYMPLECTIC6_W2 + SYMPLECTIC6_W3)
SYMPLECTIC6_WEIGHTS = (SYMPLECTIC6_W3, SYMPLECTIC6_W2, SYMPLECTIC6_W1, SYMPLECTIC6_W0,
                       SYMPLECTIC6_W1, SYMPLECTIC6_W2, SYMPLECTIC6_W3)


# Sec. 2.1: the Galactic field of Allen & Santillan (1991) in their units
# (length 1 kpc, mass 2.32e7 solar masses, velocity 10 km/s, G = 1): bulge
# M_b = 606, b_b = 0.3873; disk M_d = 3690, a_d = 5.3178, b_d = 0.25; halo
# M_h = 4615, a_h = 12, gamma = 2.02, cut at r = 100.
ALLEN_SANTILLAN = {"G": 1.0, "center": (0.0, 0.0, 0.0),
                   "m_bulge": 606.0, "b_bulge": 0.3873,
                   "m_disk": 3690.0, "a_disk": 5.3178, "b_disk": 0.25,
                   "m_halo": 4615.0, "a_halo": 12.0, "gamma": 2.02, "r_cut": 100.0}


def _ext_params(ext):
    e = dict(ALLEN_SANTILLAN)
    e.update(ext or {})
    return np.array([e["G"], *e["center"], e["m_bulge"], e["b_bulge"], e["m_disk"],
                     e["a_disk"], e["b_disk"], e["m_halo"], e["a_halo"], e["gamma"],
                     e["r_cut"]], dtype=np.float64)


def ext_field(x, ext=None, v=None):
    """Acceleration (n, 3) and potential (n,) of the external field at x,
    and with velocities v also the jerk (n, 3), d a(x + v t)/dt; ``ext``
    overrides entries of ALLEN_SANTILLAN."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))
    n = x.shape[0]
    acc = np.zeros((n, 3))
    phi = np.zeros(n)
    jerk = None
    if v is not None:
        v = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1, 3))
        jerk = np.zeros((n, 3))
    lib().orc_ext(n, _p(x), _p(v), _p(_ext_params(ext)), _p(acc), _p(jerk), _p(phi))
    return (acc, phi) if v is None else (acc, phi, jerk)


def symplectic(m, x, v, eps, dt, nsteps, order, G=1.0, weights=None, ext=None):
    """Fixed-step symplectic integration of every particle (Sec. 2.2).
    Order 2: one kick-drift-kick leapfrog step of length dt per step.
    Order 6: per step, leapfrog steps of lengths w_k dt for the seven
    weights in order (``weights`` replaces them, for tests that plant a
    wrong set).  With ``ext`` (a dict of external-field parameters, {} for
    Allen & Santillan's) the field's acceleration is added to the pair
    sum in every kick (Sec. 2.1).  Returns (x, v) after nsteps."""
    if order == 2:
        ws = (1.0,)
    elif order == 6:
        ws = SYMPLECTIC6_WEIGHTS if weights is None else tuple(weights)
    else:
        raise ValueError("order must be 2 or 6")
    x = _f64(x).copy()
    v = _f64(v).copy()

    def total_acc(xx):
        return acc(m, xx, eps, G=G) + ext_field(xx, ext)[0]

    for _ in range(int(nsteps)):
        for w in ws:
            if ext is None:
                x, v = leapfrog(m, x, v, eps, w * dt, 1, G=G)
            else:
                h = w * dt
                v = v + total_acc(x) * h / 2.0
                x = x + v * h
                v = v + total_acc(x) * h / 2.0
    return x, v


def acc_vjp(m, x, g, eps, G=1.0):
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    g = _f64(g, (n, 3))
    gx = np.zeros((n, 3))
    gm = np.zeros(n)
    lib().orc_acc_vjp(n, _p(m), _p(x), float(G), float(eps), _p(g), _p(gx), _p(gm))
    return gx, gm


def leapfrog_loss_grad(m, x0, v0, y, eps, dt, nsteps, G=1.0):
    """Returns (L, dL/dx0, dL/dv0, dL/dm) for L = sum |x(T) - y|^2."""
    m = _f64(m)
    n = m.shape[0]
    x0 = _f64(x0, (n, 3))
    v0 = _f64(v0, (n, 3))
    y = _f64(y, (n, 3))
    gx = np.zeros((n, 3))
    gv = np.zeros((n, 3))
    gm = np.zeros(n)
    L = lib().orc_leapfrog_loss_grad(n, _p(m), _p(x0), _p(v0), _p(y), float(G), float(eps),
                                     float(dt), int(nsteps), _p(gx), _p(gv), _p(gm))
    return L, gx, gv, gm


def leapfrog_adjoint_path(m, xs, lx_T, lv_T, eps, dt, G=1.0):
    """Reverse sweep along given positions xs ((nsteps+1, n, 3)); returns
    (dL/dx0, dL/dv0, dL/dm) for the terminal adjoints lx_T, lv_T."""
    m = _f64(m)
    n = m.shape[0]
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    nsteps = xs.shape[0] - 1
    lx = _f64(lx_T, (n, 3)).copy()
    lv = _f64(lv_T, (n, 3)).copy()
    lm = np.zeros(n)
    lib().orc_leapfrog_adjoint_path(n, _p(m), _p(xs), float(G), float(eps), float(dt),
                                    int(nsteps), _p(lx), _p(lv), _p(lm))
    return lx, lv, lm
