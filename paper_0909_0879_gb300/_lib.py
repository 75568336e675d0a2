"""ctypes binding of libnbody.so (the C ABI in include/nbody.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  The binding fails loudly when the library has not
been built; there is no CPU fallback.  Device-pointer calls accept any
object with ``data_ptr()`` (torch tensors) or a raw integer address.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NB_OK, NB_ERR_INVALID_ARG, NB_ERR_STATE, NB_ERR_CUDA = 0, 1, 2, 3
NB_ERR_OOM, NB_ERR_NUMERIC, NB_ERR_TIMEOUT, NB_ERR_DEVICE = 4, 5, 6, 7
NB_FP32, NB_DS = 0, 1
TICKS_LOG2 = 20
SHARD_RECORD_DOUBLES = 14  # NB_SHARD_RECORD_DOUBLES


def eps_masks(eps: float) -> int:
    """1 when the kernels zero the i == j pair explicitly: eps^2 in FP32 is
    not a normal number (the library's rule)."""
    return 1 if float(np.float32(eps * eps)) < float(np.finfo(np.float32).tiny) else 0


def _precision(p) -> int:
    if p in ("ds", NB_DS) and not isinstance(p, bool):
        return NB_DS
    if p in ("fp32", NB_FP32) and not isinstance(p, bool):
        return NB_FP32
    raise ValueError(f"precision must be 'ds', 'fp32', NB_DS or NB_FP32, not {p!r}")


class NBodyError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


class Config(C.Structure):
    _fields_ = [
        ("G", C.c_double),
        ("eps", C.c_double),
        ("eta", C.c_double),
        ("eta_start", C.c_double),
        ("lev_min", C.c_int32),
        ("lev_max", C.c_int32),
        ("precision", C.c_int32),
        ("block_steps", C.c_int32),
        ("lev_shared", C.c_int32),
        ("sync_timeout_ms", C.c_int32),
        ("stream", C.c_void_p),
    ]


class External(C.Structure):
    _fields_ = [("G", C.c_double), ("center", C.c_double * 3),
                ("m_bulge", C.c_double), ("b_bulge", C.c_double),
                ("m_disk", C.c_double), ("a_disk", C.c_double), ("b_disk", C.c_double),
                ("m_halo", C.c_double), ("a_halo", C.c_double), ("gamma_halo", C.c_double),
                ("r_cut", C.c_double)]


# (name, restype, argtypes) for every entry point in include/nbody.h
_vp, _i64, _i32, _d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
_P = C.POINTER
SIGNATURES = [
    ("nb_default_config", None, [_P(Config)]),
    ("nb_init", C.c_int, [_P(_vp), _i64, _vp, _vp, _vp, _P(Config)]),
    ("nb_destroy", None, [_vp]),
    ("nb_next_block", C.c_int, [_vp, _P(_d), _P(_i64)]),
    ("nb_predict", C.c_int, [_vp, _d]),
    ("nb_force_jerk", C.c_int, [_vp, _vp, _i64, _vp, _vp]),
    ("nb_force_jerk_dev", C.c_int, [_vp, _vp, _i64, _vp, _vp]),
    ("nb_correct", C.c_int, [_vp, _d]),
    ("nb_step", C.c_int, [_vp, _P(_d), _P(_i64)]),
    ("nb_run_blocks", C.c_int, [_vp, _d, _i64, _P(_i64), _P(_d)]),
    ("nb_set_block_mode", C.c_int, [_vp, _i32]),
    ("nb_last_block_path", C.c_int, [_vp, _P(_i32)]),
    ("nb_symplectic", C.c_int, [_vp, _i32, _d, _i64]),
    ("nb_set_symplectic_layout", C.c_int, [_vp, _i32]),
    ("nb_last_symplectic_layout", C.c_int, [_vp, _P(_i32)]),
    ("nb_external_allen_santillan", None, [_P(External)]),
    ("nb_set_external", C.c_int, [_vp, _P(External)]),
    ("nb_energy", C.c_int, [_vp, _P(_d), _P(_d), _P(_d)]),
    ("nb_get_state", C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_set_state", C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("nb_get_active", C.c_int, [_vp, _vp, _i64, _P(_i64)]),
    ("nb_relayout", C.c_int, [_vp]),
    ("nb_set_relayout_every", C.c_int, [_vp, _i64]),
    ("nb_get_storage_order", C.c_int, [_vp, _vp, _P(_i64)]),
    ("nb_get_counters", C.c_int, [_vp, _P(_i64), _P(_i64), _P(_i64)]),
    ("nb_sync", C.c_int, [_vp]),
    ("nb_launch_count", _i64, [_vp]),
    ("nb_set_force_variant", C.c_int, [_vp, _i32, _i32]),
    ("nb_spatial_order", C.c_int, [_i64, _vp, _i64, _vp]),
    ("nb_set_force_table", C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    ("nb_variant_info", C.c_int, [_i32, _P(_i32), _P(_i32), _P(_i32), _P(_i32), _P(_i32)]),
    ("nb_debug_inject", C.c_int, [_vp, _i32]),
    ("nb_batched_init", C.c_int, [_P(_vp), _i32, _vp, _vp, _vp, _vp, _P(Config)]),
    ("nb_batched_destroy", None, [_vp]),
    ("nb_batched_run", C.c_int, [_vp, _i64]),
    ("nb_batched_run_per_cluster", C.c_int, [_vp, _i64]),
    ("nb_batched_set_tuning", C.c_int, [_vp, _i32, _i32, _i32, _i32]),
    ("nb_batched_variant_info", C.c_int, [_i32, _P(_i32), _P(_i32), _P(_i32), _P(_i32)]),
    ("nb_batched_energy", C.c_int, [_vp, _vp, _vp]),
    ("nb_batched_get_state", C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("nb_batched_sync", C.c_int, [_vp]),
    ("nb_batched_launch_count", _i64, [_vp]),
    ("nb_lf_acc", C.c_int, [_i64, _vp, _vp, C.c_float, C.c_float, _vp, _vp]),
    ("nb_lf_acc_vjp", C.c_int, [_i64, _vp, _vp, _vp, C.c_float, C.c_float, _vp, _vp, _vp]),
    ("nb_lf_ckpt_floats", _i64, [_i64, _i64, _i32]),
    ("nb_lf_work_floats", _i64, [_i64, _i32]),
    ("nb_lf_forward", C.c_int, [_i64, _vp, _vp, _vp, _vp, _i64, C.c_float, C.c_float,
                                C.c_float, _i32, _vp, _vp]),
    ("nb_lf_backward", C.c_int, [_i64, _vp, _vp, _i64, C.c_float, C.c_float, C.c_float, _i32,
                                 _vp, _vp, _vp, _vp, _vp]),
    ("nb_shard_set", C.c_int, [_vp, _i32, _i32, _vp]),
    ("nb_shard_offsets", C.c_int, [_vp, _vp]),
    ("nb_shard_export", C.c_int, [_vp, _vp, _P(_i64)]),
    ("nb_shard_import", C.c_int, [_vp, _vp, _i64]),
    ("nb_force_jerk_noalloc", C.c_int, [_i64, _vp, _vp, _vp, _vp, _i64, _d, _d, _i32, _vp,
                                         _vp, _vp]),
    ("nb_status_string", C.c_char_p, [C.c_int]),
    ("nb_last_error", C.c_char_p, []),
]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libnbody.so (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(
                f"libnbody.so is not built ({path}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        _build.build()
    L = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != NB_OK:
        L = load()
        raise NBodyError(status, L.nb_last_error().decode(errors="replace"))


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(a)}")


def _f64(a, shape):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(shape)


def variant_info(v: int):
    L = load()
    p, i, t, n, k = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(L.nb_variant_info(v, C.byref(p), C.byref(i), C.byref(t), C.byref(n), C.byref(k)))
    return {"precision": p.value, "ipt": i.value, "tpi": t.value, "threads": n.value,
            "packed": k.value}


def num_variants() -> int:
    v = 0
    L = load()
    while L.nb_variant_info(v, None, None, None, None, None) == NB_OK:
        v += 1
    return v


def spatial_order(x, leaf: int = 256) -> np.ndarray:
    """Permutation (int64) that stores particles leaf by leaf of a balanced
    bisection tree (see nb_spatial_order in include/nbody.h)."""
    x = _f64(x, (-1, 3))
    perm = np.zeros(x.shape[0], dtype=np.int64)
    _check(load().nb_spatial_order(x.shape[0], x.ctypes.data, int(leaf),
                                   perm.ctypes.data if x.shape[0] else None))
    return perm


def default_config() -> Config:
    cfg = Config()
    load().nb_default_config(C.byref(cfg))
    return cfg


class NBody:
    """A direct-summation N-body system on the GPU (one libnbody context).

    Host arrays are float64 numpy arrays: m (n,), x and v (n, 3).
    """

    def __init__(self, m, x, v, *, G=1.0, eps=1e-3, eta=0.01, eta_start=0.01,
                 lev_min=3, lev_max=20, precision="ds", block_steps=True,
                 lev_shared=8, stream=None, sync_timeout_ms=0):
        L = load()
        m = np.ascontiguousarray(m, dtype=np.float64)
        n = m.shape[0]
        x = _f64(x, (n, 3))
        v = _f64(v, (n, 3))
        cfg = default_config()
        cfg.G, cfg.eps, cfg.eta, cfg.eta_start = float(G), float(eps), float(eta), float(eta_start)
        cfg.lev_min, cfg.lev_max = int(lev_min), int(lev_max)
        cfg.precision = _precision(precision)
        cfg.block_steps = 1 if block_steps else 0
        cfg.lev_shared = int(lev_shared)
        cfg.sync_timeout_ms = int(sync_timeout_ms)
        if stream is None:
            cfg.stream = None
        elif hasattr(stream, "cuda_stream"):  # torch.cuda.Stream
            cfg.stream = stream.cuda_stream or None
        else:
            cfg.stream = int(stream) or None
        self.cfg = cfg
        self.n = n
        h = C.c_void_p()
        _check(L.nb_init(C.byref(h), n, m.ctypes.data, x.ctypes.data, v.ctypes.data,
                         C.byref(cfg)))
        self._h = h
        self._L = L

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.nb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- integrator
    def next_block(self):
        t, na = C.c_double(), C.c_int64()
        _check(self._L.nb_next_block(self._h, C.byref(t), C.byref(na)))
        return t.value, na.value

    def predict(self, t: float):
        _check(self._L.nb_predict(self._h, float(t)))

    def force_jerk(self, idx=None, n_idx: int = -1):
        """Host path: returns (acc, jerk) numpy arrays of shape (n_idx, 3)."""
        if idx is None:
            if n_idx < 0:
                _, cnt = self.active_count()
            else:
                cnt = n_idx
            acc = np.zeros((cnt, 3))
            jerk = np.zeros((cnt, 3))
            _check(self._L.nb_force_jerk(self._h, None, cnt, acc.ctypes.data, jerk.ctypes.data))
            return acc, jerk
        ii = np.ascontiguousarray(idx, dtype=np.int32)
        acc = np.zeros((ii.shape[0], 3))
        jerk = np.zeros((ii.shape[0], 3))
        _check(self._L.nb_force_jerk(self._h, ii.ctypes.data if ii.size else None, ii.shape[0],
                                     acc.ctypes.data, jerk.ctypes.data))
        return acc, jerk

    def force_jerk_dev(self, d_idx, n_idx: int, d_acc, d_jerk):
        """Device path, asynchronous on the context stream."""
        _check(self._L.nb_force_jerk_dev(self._h, _ptr(d_idx), int(n_idx), _ptr(d_acc),
                                         _ptr(d_jerk)))

    def correct(self, t: float):
        _check(self._L.nb_correct(self._h, float(t)))

    def step(self):
        t, na = C.c_double(), C.c_int64()
        _check(self._L.nb_step(self._h, C.byref(t), C.byref(na)))
        return t.value, na.value

    def run_blocks(self, t_end: float, max_blocks: int = 0):
        """Device-resident block steps until t_end (graph replays); returns
        (block steps taken, time of the last block)."""
        nb, tl = C.c_int64(), C.c_double()
        _check(self._L.nb_run_blocks(self._h, float(t_end), int(max_blocks), C.byref(nb),
                                     C.byref(tl)))
        return nb.value, tl.value

    BLOCK_MODES = {"auto": 0, "general": 1}

    def set_block_mode(self, mode: str):
        """'auto': fused device-resident steps when the schedule allows them;
        'general': always the general scheduler."""
        _check(self._L.nb_set_block_mode(self._h, self.BLOCK_MODES[mode]))

    def last_block_path(self) -> str:
        """'fused' or 'general': the form the last run_blocks call ran."""
        f = C.c_int32()
        _check(self._L.nb_last_block_path(self._h, C.byref(f)))
        return "fused" if f.value else "general"

    def symplectic(self, order: int, dt: float, nsteps: int):
        """Fixed-step symplectic integration of every particle: order 2
        (kick-drift-kick leapfrog) or 6 (seven-stage composition), nsteps
        steps of dt.  Afterwards x, v and a (= A(x)) are current; Hermite
        calls need set_state first."""
        _check(self._L.nb_symplectic(self._h, int(order), float(dt), int(nsteps)))

    SYMPLECTIC_LAYOUTS = {"auto": 0, "as_given": 1, "spatial": 2}

    def set_symplectic_layout(self, mode: str):
        """'auto', 'as_given' or 'spatial': the particle order symplectic
        runs step in (the state is returned in the caller's order)."""
        _check(self._L.nb_set_symplectic_layout(self._h, self.SYMPLECTIC_LAYOUTS[mode]))

    def last_symplectic_layout(self) -> str:
        f = C.c_int32()
        _check(self._L.nb_last_symplectic_layout(self._h, C.byref(f)))
        return "spatial" if f.value else "as_given"

    def set_external(self, ext=None):
        """Set the external Galactic field (a dict of nb_external fields,
        missing ones from Allen & Santillan's model; {} for that model
        itself) or remove it (None)."""
        if ext is None:
            _check(self._L.nb_set_external(self._h, None))
            return
        e = External()
        self._L.nb_external_allen_santillan(C.byref(e))
        for k, val in ext.items():
            if k == "center":
                e.center[:] = [float(c) for c in val]
            elif k == "gamma":
                e.gamma_halo = float(val)
            else:
                setattr(e, k, float(val))
        _check(self._L.nb_set_external(self._h, C.byref(e)))

    def run_until(self, t_end: float):
        """Block steps until every particle has reached t_end (a tick multiple
        reachable by the largest step).  Returns the number of block steps."""
        steps = 0
        tick_end = int(round(t_end * 2**TICKS_LOG2))
        while True:
            st = self.get_state(want=("t_tick", "lev"))
            due = st["t_tick"] + (1 << (TICKS_LOG2 - st["lev"].astype(np.int64)))
            if due.min() > tick_end:
                return steps
            self.step()
            steps += 1

    def energy(self):
        k, w, e = C.c_double(), C.c_double(), C.c_double()
        _check(self._L.nb_energy(self._h, C.byref(k), C.byref(w), C.byref(e)))
        return k.value, w.value, e.value

    _STATE_SPEC = {"x": (3, np.float64), "v": (3, np.float64), "a": (3, np.float64),
                   "jerk": (3, np.float64), "t_tick": (0, np.int64), "lev": (0, np.int32)}

    def get_state(self, want=("x", "v", "a", "jerk", "t_tick", "lev"), out=None):
        """Copy the state to host arrays.  With out (a dict of C-contiguous
        arrays of the right shapes and dtypes, e.g. in pinned memory, as a
        previous get_state returned) the copies land in those arrays and no
        host memory is allocated or first touched."""
        n = self.n
        bufs = {}
        res = {}
        for key, (w, dt) in self._STATE_SPEC.items():
            if key not in want:
                continue
            shape = (n, w) if w else (n,)
            if out is not None and key in out:
                a = out[key]
                if a.shape != shape or a.dtype != dt or not a.flags.c_contiguous:
                    raise ValueError(f"out[{key!r}] must be a C-contiguous {dt.__name__} "
                                     f"array of shape {shape}")
            else:
                a = np.zeros(shape, dtype=dt)
            bufs[key] = res[key] = a
        out = res
        p = {k: (bufs[k].ctypes.data if k in bufs else None)
             for k in ("x", "v", "a", "jerk", "t_tick", "lev")}
        _check(self._L.nb_get_state(self._h, p["x"], p["v"], p["a"], p["jerk"], p["t_tick"],
                                    p["lev"]))
        return out

    def set_state(self, st):
        n = self.n
        x = _f64(st["x"], (n, 3))
        v = _f64(st["v"], (n, 3))
        a = _f64(st["a"], (n, 3))
        jk = _f64(st["jerk"], (n, 3))
        t = np.ascontiguousarray(st["t_tick"], dtype=np.int64)
        lev = np.ascontiguousarray(st["lev"], dtype=np.int32)
        _check(self._L.nb_set_state(self._h, x.ctypes.data, v.ctypes.data, a.ctypes.data,
                                    jk.ctypes.data, t.ctypes.data, lev.ctypes.data))

    def active_count(self):
        na = C.c_int64()
        _check(self._L.nb_get_active(self._h, None, 0, C.byref(na)))
        return None, na.value

    def active(self):
        _, cnt = self.active_count()
        idx = np.zeros(max(cnt, 1), dtype=np.int32)
        na = C.c_int64()
        _check(self._L.nb_get_active(self._h, idx.ctypes.data, idx.shape[0], C.byref(na)))
        return idx[: na.value].copy()

    def relayout(self):
        """Re-store the particles in a bisection order of their current
        positions (the caller's order of every input and output stays)."""
        _check(self._L.nb_relayout(self._h))

    def set_relayout_every(self, block_steps: int):
        """Relayout automatically after this many block steps (0: off)."""
        _check(self._L.nb_set_relayout_every(self._h, int(block_steps)))

    def storage_order(self):
        """(perm, relayouts): perm[s] is the caller's index of the particle
        stored in slot s."""
        perm = np.zeros(self.n, dtype=np.int32)
        cnt = C.c_int64()
        _check(self._L.nb_get_storage_order(self._h, perm.ctypes.data, C.byref(cnt)))
        return perm, cnt.value

    def counters(self):
        b, i, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._L.nb_get_counters(self._h, C.byref(b), C.byref(i), C.byref(c)))
        return {"blocks": b.value, "interactions": i.value, "clamped": c.value}

    def sync(self):
        _check(self._L.nb_sync(self._h))

    def launch_count(self) -> int:
        return int(self._L.nb_launch_count(self._h))

    def set_force_variant(self, variant: int = -1, grid_ctas: int = 0):
        _check(self._L.nb_set_force_variant(self._h, int(variant), int(grid_ctas)))

    def set_force_table(self, table):
        """table: list of (min_active, variant) or (min_active, variant,
        grid_cap), checked in order (grid_cap 0: the full persistent
        grid)."""
        mins = np.ascontiguousarray([t[0] for t in table], dtype=np.int64)
        vars_ = np.ascontiguousarray([t[1] for t in table], dtype=np.int32)
        grids = np.ascontiguousarray([t[2] if len(t) > 2 else 0 for t in table], dtype=np.int32)
        k = len(table)
        _check(self._L.nb_set_force_table(self._h, k, mins.ctypes.data if k else None,
                                          vars_.ctypes.data if k else None,
                                          grids.ctypes.data if k else None))

    # -- i-split shards (see nb_shard_set in include/nbody.h)
    def shard_set(self, nranks: int, rank: int, bounds=None):
        """Make this context shard `rank` of `nranks` owning particles
        [bounds[rank], bounds[rank + 1]) (nranks == 1: unsharded)."""
        self._shards = int(nranks)
        if nranks == 1:
            _check(self._L.nb_shard_set(self._h, 1, 0, None))
            return
        b = np.ascontiguousarray(bounds, dtype=np.int64)
        _check(self._L.nb_shard_set(self._h, int(nranks), int(rank), b.ctypes.data))

    def shard_offsets(self) -> np.ndarray:
        """Offsets of every rank's slice in the current block's active list
        (nranks + 1 entries)."""
        out = np.zeros(getattr(self, "_shards", 1) + 1, dtype=np.int64)
        _check(self._L.nb_shard_offsets(self._h, out.ctypes.data))
        return out

    def shard_export(self, d_rec) -> int:
        """Corrected records of the own slice into device memory d_rec
        (rows of SHARD_RECORD_DOUBLES doubles); returns the row count."""
        cnt = C.c_int64()
        _check(self._L.nb_shard_export(self._h, _ptr(d_rec), C.byref(cnt)))
        return cnt.value

    def shard_import(self, d_rec, n_rec: int):
        """The whole active list's records (list order) from device memory."""
        _check(self._L.nb_shard_import(self._h, _ptr(d_rec), int(n_rec)))

    def inject(self, kind: int):
        _check(self._L.nb_debug_inject(self._h, int(kind)))


def batched_variant_info(v: int):
    L = load()
    p, i, t, k = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(L.nb_batched_variant_info(v, C.byref(p), C.byref(i), C.byref(t), C.byref(k)))
    return {"precision": p.value, "ipt": i.value, "threads": t.value, "packed": k.value}


def num_batched_variants() -> int:
    v = 0
    L = load()
    while L.nb_batched_variant_info(v, None, None, None, None) == NB_OK:
        v += 1
    return v


class Batch:
    """Many independent clusters advanced together with a shared step
    (one libnbody batched context).  ``offsets`` has n_clusters + 1 entries;
    cluster c is particles offsets[c]:offsets[c+1] of m, x, v."""

    def __init__(self, offsets, m, x, v, *, G=1.0, eps=1e-3, lev_shared=8, precision="ds",
                 stream=None):
        L = load()
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        m = np.ascontiguousarray(m, dtype=np.float64)
        n = m.shape[0]
        x = _f64(x, (n, 3))
        v = _f64(v, (n, 3))
        cfg = default_config()
        cfg.G, cfg.eps = float(G), float(eps)
        cfg.block_steps = 0
        cfg.lev_shared = int(lev_shared)
        cfg.precision = _precision(precision)
        if stream is not None:
            cfg.stream = (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)) or None
        self.n_clusters = off.shape[0] - 1
        self.n = n
        self.offsets = off
        self.precision = cfg.precision
        self.mask = eps_masks(cfg.eps)
        h = C.c_void_p()
        _check(L.nb_batched_init(C.byref(h), self.n_clusters, off.ctypes.data, m.ctypes.data,
                                 x.ctypes.data, v.ctypes.data, C.byref(cfg)))
        self._h = h
        self._L = L

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.nb_batched_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, nsteps: int):
        _check(self._L.nb_batched_run(self._h, int(nsteps)))

    def run_per_cluster(self, nsteps: int):
        _check(self._L.nb_batched_run_per_cluster(self._h, int(nsteps)))

    def set_tuning(self, variant=-1, steps_per_launch=1000, grid_ctas=0, use_graph=True):
        _check(self._L.nb_batched_set_tuning(self._h, int(variant), int(steps_per_launch),
                                             int(grid_ctas), 1 if use_graph else 0))

    def energy(self):
        k = np.zeros(self.n_clusters)
        w = np.zeros(self.n_clusters)
        _check(self._L.nb_batched_energy(self._h, k.ctypes.data, w.ctypes.data))
        return k, w

    def get_state(self):
        out = {k: np.zeros((self.n, 3)) for k in ("x", "v", "a", "jerk")}
        _check(self._L.nb_batched_get_state(self._h, out["x"].ctypes.data, out["v"].ctypes.data,
                                            out["a"].ctypes.data, out["jerk"].ctypes.data))
        return out

    def sync(self):
        _check(self._L.nb_batched_sync(self._h))

    def launch_count(self) -> int:
        return int(self._L.nb_batched_launch_count(self._h))


def force_jerk_noalloc(n, d_m, d_x, d_v, d_idx, n_idx, d_acc, d_jerk, *, eps, G=1.0,
                       precision="ds", stream=None):
    """Allocation-free force + jerk on caller-owned device arrays (see
    nb_force_jerk_noalloc in include/nbody.h).  Asynchronous on ``stream``
    (a torch stream, a raw handle, or None for the default stream)."""
    L = load()
    if stream is None:
        sp = None
    elif hasattr(stream, "cuda_stream"):
        sp = stream.cuda_stream or None
    else:
        sp = int(stream) or None
    prec = _precision(precision)
    _check(L.nb_force_jerk_noalloc(int(n), _ptr(d_m), _ptr(d_x), _ptr(d_v), _ptr(d_idx),
                                   int(n_idx), float(eps), float(G), prec, _ptr(d_acc),
                                   _ptr(d_jerk), sp))


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or None
    return int(stream) or None


def lf_acc(n, d_x, d_m, d_acc, *, eps, G=1.0, stream=None):
    _check(load().nb_lf_acc(int(n), _ptr(d_x), _ptr(d_m), float(eps), float(G), _ptr(d_acc),
                            _stream_ptr(stream)))


def lf_acc_vjp(n, d_x, d_m, d_g, d_gx, d_gm, *, eps, G=1.0, stream=None):
    _check(load().nb_lf_acc_vjp(int(n), _ptr(d_x), _ptr(d_m), _ptr(d_g), float(eps), float(G),
                                _ptr(d_gx), _ptr(d_gm), _stream_ptr(stream)))


def lf_ckpt_floats(n, nsteps, ckpt_every) -> int:
    return int(load().nb_lf_ckpt_floats(int(n), int(nsteps), int(ckpt_every)))


def lf_work_floats(n, ckpt_every) -> int:
    return int(load().nb_lf_work_floats(int(n), int(ckpt_every)))


def lf_forward(n, d_m, d_x, d_v, d_acc, nsteps, dt, d_ckpt, *, eps, G=1.0, ckpt_every=8,
               stream=None):
    _check(load().nb_lf_forward(int(n), _ptr(d_m), _ptr(d_x), _ptr(d_v), _ptr(d_acc),
                                int(nsteps), float(dt), float(eps), float(G), int(ckpt_every),
                                _ptr(d_ckpt), _stream_ptr(stream)))


def lf_backward(n, d_m, d_ckpt, nsteps, dt, d_lx, d_lv, d_lm, d_work, *, eps, G=1.0,
                ckpt_every=8, stream=None):
    _check(load().nb_lf_backward(int(n), _ptr(d_m), _ptr(d_ckpt), int(nsteps), float(dt),
                                 float(eps), float(G), int(ckpt_every), _ptr(d_lx), _ptr(d_lv),
                                 _ptr(d_lm), _ptr(d_work), _stream_ptr(stream)))
