"""GPU parity of the batched form (many independent clusters, shared-step
Hermite-4, persistent kernel under a CUDA graph) against the FP64 oracle run
cluster by cluster, plus its bitwise invariances."""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    return _lib


def make_clusters(n_clusters, seed, lo=16, hi=1024):
    sizes = ics.cluster_sizes(n_clusters, seed, lo, hi)
    ms, xs, vs = [], [], []
    for c, nc in enumerate(sizes):
        m, x, v = ics.plummer(int(nc), (seed, c))
        ms.append(m); xs.append(x); vs.append(v)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return off, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs)


def test_batched_vs_oracle_per_cluster(nb, oracle_mod):
    """24 clusters (16..1024 bodies), eps = 1e-3, dt = 1/256, 64 steps:
    per-cluster energy error within 2x the oracle's, positions close."""
    off, m, x, v = make_clusters(24, 1004)
    eps, lev, steps = 1e-3, 8, 64
    with nb.Batch(off, m, x, v, eps=eps, lev_shared=lev) as b:
        k0, w0 = b.energy()
        b.run(steps)
        st = b.get_state()
        k1, w1 = b.energy()
    bad = []
    for c in range(len(off) - 1):
        s = slice(off[c], off[c + 1])
        E0o = oracle_mod.energy(m[s], x[s], v[s], eps)[2]
        assert abs(k0[c] + w0[c] - E0o) <= 1e-12 * abs(E0o)
        xo, vo, _, _ = oracle_mod.hermite_shared(m[s], x[s], v[s], eps, lev, steps)
        dEo = abs(oracle_mod.energy(m[s], xo, vo, eps)[2] - E0o) / abs(E0o)
        dEg = abs(k1[c] + w1[c] - E0o) / abs(E0o)
        if dEg > 2 * max(dEo, 1e-10):
            bad.append((c, off[c + 1] - off[c], dEg, dEo))
    assert not bad, bad


def test_batched_positions_track_oracle_short(nb, oracle_mod):
    off, m, x, v = make_clusters(12, 77)
    eps, lev = 1e-3, 8
    with nb.Batch(off, m, x, v, eps=eps, lev_shared=lev) as b:
        b.run(4)
        st = b.get_state()
    for c in range(len(off) - 1):
        s = slice(off[c], off[c + 1])
        xo, vo, ao, jo = oracle_mod.hermite_shared(m[s], x[s], v[s], eps, lev, 4)
        assert np.abs(st["x"][s] - xo).max() < 1e-9
        assert np.abs(st["v"][s] - vo).max() < 1e-7


def test_batched_modes_bitwise_equal(nb):
    """Persistent + graph, persistent without graph, per-cluster launches,
    and a cluster run alone all give bit-identical states."""
    off, m, x, v = make_clusters(40, 5)
    steps = 7
    res = []
    for mode in ("graph", "plain", "per_cluster"):
        with nb.Batch(off, m, x, v, eps=1e-3, lev_shared=8) as b:
            b.set_tuning(-1, 3, 0, mode == "graph")
            if mode == "per_cluster":
                b.run_per_cluster(steps)
            else:
                b.run(steps)
            res.append(b.get_state())
    for r in res[1:]:
        for k in r:
            assert np.array_equal(r[k], res[0][k]), k
    c = 17
    s = slice(off[c], off[c + 1])
    with nb.Batch(np.array([0, off[c + 1] - off[c]]), m[s], x[s], v[s], eps=1e-3, lev_shared=8) as b:
        b.run(steps)
        alone = b.get_state()
    for k in alone:
        assert np.array_equal(alone[k], res[0][k][s]), k


def test_batched_every_variant(nb, oracle_mod):
    off, m, x, v = make_clusters(10, 9)
    ref = None
    for var in range(nb.num_batched_variants()):
        info = nb.batched_variant_info(var)
        prec = "ds" if info["precision"] else "fp32"
        with nb.Batch(off, m, x, v, eps=1e-3, lev_shared=8, precision=prec) as b:
            try:
                b.set_tuning(var, 5, 0, True)
            except nb.NBodyError:
                continue
            b.run(10)
            st = b.get_state()
        if ref is None:
            ref = {}
            for c in range(len(off) - 1):
                s = slice(off[c], off[c + 1])
                ref[c] = oracle_mod.hermite_shared(m[s], x[s], v[s], 1e-3, 8, 10)[0]
        tol = 1e-8 if prec == "ds" else 1e-5
        for c in range(len(off) - 1):
            s = slice(off[c], off[c + 1])
            assert np.abs(st["x"][s] - ref[c]).max() < tol, (var, c)
