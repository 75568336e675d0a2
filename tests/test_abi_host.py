"""CPU-only checks of the C ABI library: it builds, loads, exports every
entry point declared in include/nbody.h, and its host-side validation works
without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0909_0879_gb300 import build, _lib

    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nbody.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), f"{name} declared in nbody.h but not exported"


def test_binding_covers_every_declared_symbol():
    from paper_0909_0879_gb300 import _lib

    bound = {s[0] for s in _lib.SIGNATURES}
    assert bound == set(declared_functions())


def test_status_strings_and_default_config(lib):
    from paper_0909_0879_gb300 import _lib

    assert lib.nb_status_string(0) == b"ok"
    assert lib.nb_status_string(6) == b"watchdog timeout"
    cfg = _lib.default_config()
    assert cfg.G == 1.0 and cfg.precision == 1 and cfg.lev_min == 3 and cfg.lev_max == 20


def test_variant_table(lib):
    from paper_0909_0879_gb300 import _lib

    n = _lib.num_variants()
    assert n >= 10
    infos = [_lib.variant_info(v) for v in range(n)]
    assert {i["precision"] for i in infos} == {0, 1}
    for i in infos:
        assert i["threads"] % i["tpi"] == 0 and 32 % i["tpi"] == 0 or i["tpi"] <= 32
    with pytest.raises(_lib.NBodyError) as e:
        _lib.variant_info(n)
    assert e.value.status == _lib.NB_ERR_INVALID_ARG


def test_init_rejects_bad_arguments_before_any_device_call(lib):
    """Validation happens on the host, so these fail the same way with or
    without a GPU."""
    from paper_0909_0879_gb300 import _lib

    m = np.ones(4) / 4
    x = np.random.default_rng(0).normal(size=(4, 3))
    v = np.zeros((4, 3))
    cases = [
        dict(m=m[:0], x=x[:0], v=v[:0]),                 # n = 0
        dict(m=m, x=np.where(x > 0, np.nan, x), v=v),    # non-finite
        dict(m=-m, x=x, v=v),                            # negative mass
    ]
    for c in cases:
        with pytest.raises(_lib.NBodyError) as e:
            _lib.NBody(c["m"], c["x"], c["v"])
        assert e.value.status == _lib.NB_ERR_INVALID_ARG
    for kw in (dict(eps=-1.0), dict(lev_min=5, lev_max=4), dict(lev_max=21), dict(G=0.0),
               dict(eta=0.0), dict(block_steps=False, lev_shared=25)):
        with pytest.raises(_lib.NBodyError) as e:
            _lib.NBody(m, x, v, **kw)
        assert e.value.status == _lib.NB_ERR_INVALID_ARG, kw
    h = C.c_void_p()
    assert lib.nb_init(C.byref(h), 4, None, None, None, None) == _lib.NB_ERR_INVALID_ARG
    assert b"null" in lib.nb_last_error()
    assert lib.nb_debug_inject(None, 9) == _lib.NB_ERR_INVALID_ARG
    assert lib.nb_debug_inject(None, 2) == _lib.NB_ERR_INVALID_ARG
    lib.nb_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_0909_0879_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_spatial_order_is_a_balanced_tree_layout(lib):
    """Host-only helper: a permutation whose 256-particle leaves are compact
    and balanced, deterministic for the same input."""
    from paper_0909_0879_gb300 import _lib, ics

    m, x, v = ics.king(10000, 7.0, 3)
    p = _lib.spatial_order(x, 256)
    assert np.array_equal(np.sort(p), np.arange(10000))
    assert np.array_equal(p, _lib.spatial_order(x, 256))
    xs = x[p]
    # leaf boxes are far smaller than those of the unordered particles
    tiles = [np.ptp(xs[k:k + 256], axis=0).max() for k in range(0, 9984, 256)]
    raw = [np.ptp(x[k:k + 256], axis=0).max() for k in range(0, 9984, 256)]
    assert np.median(tiles) < 0.6 * np.median(raw)
    # uniform points: each leaf's box holds about its share of the volume
    u = np.random.default_rng(1).uniform(0, 1, (65536, 3))
    pu = _lib.spatial_order(u, 256)
    vol = [np.prod(np.ptp(u[pu[k:k + 256]], axis=0)) for k in range(0, 65536, 256)]
    assert np.mean(vol) < 2.0 * 256 / 65536
    # a set of the same points in another order gives the same leaf sets
    q = np.random.default_rng(0).permutation(10000)
    p2 = _lib.spatial_order(x[q], 256)
    assert sorted(map(tuple, np.sort(q[p2][: 9984].reshape(-1, 256), axis=1))) == \
        sorted(map(tuple, np.sort(p[: 9984].reshape(-1, 256), axis=1)))
    with pytest.raises(_lib.NBodyError):
        _lib.spatial_order(np.full((3, 3), np.nan), 256)
    # large sets split their upper levels over threads: the same permutation
    # every time, and every 256-record leaf compact along a bisection
    big = np.random.default_rng(2).normal(0.0, 1.0, (300000, 3))
    pb = _lib.spatial_order(big, 256)
    assert np.array_equal(np.sort(pb), np.arange(300000))
    for _ in range(3):
        assert np.array_equal(pb, _lib.spatial_order(big, 256))
    leaf_ext = np.ptp(big[pb[: 299776]].reshape(-1, 256, 3), axis=1).max(axis=1)
    assert np.median(leaf_ext) < 0.2 * np.ptp(big, axis=0).max()
