"""The allocation-free entry point, nb_force_jerk_noalloc, through the C ABI.

It serves callers that cannot let a library allocate device memory (their
memory belongs to another allocator, or an allocation's possible device
synchronisation is not allowed); its only scratch is a fixed static device
array.  The test checks two calls in a row against the context-based entry
point nb_force_jerk_dev on the same particles, within the split-precision
tolerance the parity tests use (1e-6 for the acceleration, 1e-5 for the
jerk, norm-wise and relative to each sum's condition).  This file is named
to be collected last.
"""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu


def _compare(acc, jerk, ref_a, ref_j, cond, tol_a, tol_j):
    na = np.linalg.norm(acc - ref_a) / np.linalg.norm(ref_a)
    nj = np.linalg.norm(jerk - ref_j) / np.linalg.norm(ref_j)
    ca = (np.linalg.norm(acc - ref_a, axis=1) / cond[0]).max()
    cj = (np.linalg.norm(jerk - ref_j, axis=1) / cond[1]).max()
    assert na <= tol_a and ca <= tol_a, (na, ca)
    assert nj <= tol_j and cj <= tol_j, (nj, cj)


def test_noalloc_matches_context_entry_point(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    n, eps = 5003, 1e-3
    m, x, v = ics.plummer(n, 4242, masses=ics.salpeter_masses(n, 4242))
    dev = torch.device("cuda", 0)
    d_m = torch.from_numpy(m).to(dev)
    d_x = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    d_v = torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    cases = [ics.random_active_subset(n, 1700, 7), np.arange(n, dtype=np.int32)]
    for prec in ("ds", "fp32"):
        tol_a, tol_j = (1e-6, 1e-5) if prec == "ds" else (1e-3, 1e-3)
        with _lib.NBody(m, x, v, eps=eps, precision=prec) as s:
            for call, idx in enumerate(cases):
                n_idx = len(idx)
                d_idx = torch.from_numpy(idx).to(dev)
                ref_a = torch.zeros((n_idx, 3), dtype=torch.float64, device=dev)
                ref_j = torch.zeros_like(ref_a)
                s.force_jerk_dev(d_idx, n_idx, ref_a, ref_j)
                s.sync()
                acc = torch.full((n_idx, 3), float("nan"), dtype=torch.float64, device=dev)
                jerk = torch.full_like(acc, float("nan"))
                # the second call passes no index list (identity order)
                _lib.force_jerk_noalloc(n, d_m, d_x, d_v, d_idx if call == 0 else None, n_idx,
                                        acc, jerk, eps=eps, precision=prec)
                torch.cuda.synchronize(dev)
                cond = oracle_mod.force_jerk_abs(m, x, v, eps, idx=idx)
                _compare(acc.cpu().numpy(), jerk.cpu().numpy(), ref_a.cpu().numpy(),
                         ref_j.cpu().numpy(), cond, tol_a, tol_j)


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    d = torch.zeros(30, dtype=torch.float64, device="cuda")
    for n, n_idx in ((0, 1), (10, -1), (10, 11), (2**31, 1)):
        with pytest.raises(_lib.NBodyError) as e:
            _lib.force_jerk_noalloc(n, d, d, d, None, n_idx, d, d, eps=1e-3)
        assert e.value.status == _lib.NB_ERR_INVALID_ARG
