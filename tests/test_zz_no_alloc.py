"""The allocation-free entry point, nb_force_jerk_noalloc, through the C ABI.

It serves callers that cannot let a library allocate device memory (their
memory belongs to another allocator, or an allocation's possible device
synchronisation is not allowed); its only scratch is a fixed static device
array.  Every case makes two calls in a row and checks them

  * against the FP64 oracle on the same particles, within the tolerance of
    the parity tests: split precision 1e-6 for the acceleration and 1e-5
    for the jerk, norm-wise and relative to each sum's condition
    sum_j |f_ij| (FP32 positions: 1e-3), and
  * against the context-based entry point nb_force_jerk_dev, within the
    same tolerance.

The cases reach every output path of the kernel: i-blocks split across
CTAs (partial sums in the static array, then the fix-up kernel), i-blocks
written directly by the one CTA that covers them, launches where every CTA
covers whole i-blocks (the fix-up kernel is skipped), and the eps == 0
kernels that zero the i == j term.  This file is named to be collected
last.
"""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"ds": (1e-6, 1e-5), "fp32": (1e-3, 1e-3)}


def _within(acc, jerk, ref_a, ref_j, cond, prec, what):
    tol_a, tol_j = TOL[prec]
    na = np.linalg.norm(acc - ref_a) / np.linalg.norm(ref_a)
    nj = np.linalg.norm(jerk - ref_j) / np.linalg.norm(ref_j)
    ca = (np.linalg.norm(acc - ref_a, axis=1) / cond[0]).max()
    cj = (np.linalg.norm(jerk - ref_j, axis=1) / cond[1]).max()
    assert na <= tol_a and ca <= tol_a, (what, prec, "acc", na, ca)
    assert nj <= tol_j and cj <= tol_j, (what, prec, "jerk", nj, cj)


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    return torch, _lib, torch.device("cuda", 0)


def _run_case(cuda, oracle_mod, m, x, v, eps, idx_list, precs=("ds", "fp32"),
              pass_idx=(True, True)):
    """Two no-alloc calls per precision (the index lists idx_list[0] and
    [1]); each against the oracle and against nb_force_jerk_dev."""
    torch, _lib, dev = cuda
    n = len(m)
    d_m = torch.from_numpy(m).to(dev)
    d_x = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    d_v = torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    refs = []
    for idx in idx_list:
        ra, rj = oracle_mod.force_jerk(m, x, v, eps, idx=idx)
        cond = oracle_mod.force_jerk_abs(m, x, v, eps, idx=idx)
        refs.append((ra, rj, cond))
    for prec in precs:
        with _lib.NBody(m, x, v, eps=eps, precision=prec) as s:
            for call, (idx, (ra, rj, cond)) in enumerate(zip(idx_list, refs)):
                n_idx = len(idx)
                d_idx = torch.from_numpy(idx).to(dev)
                ctx_a = torch.zeros((n_idx, 3), dtype=torch.float64, device=dev)
                ctx_j = torch.zeros_like(ctx_a)
                s.force_jerk_dev(d_idx, n_idx, ctx_a, ctx_j)
                s.sync()
                acc = torch.full((n_idx, 3), float("nan"), dtype=torch.float64, device=dev)
                jerk = torch.full_like(acc, float("nan"))
                _lib.force_jerk_noalloc(n, d_m, d_x, d_v, d_idx if pass_idx[call] else None,
                                        n_idx, acc, jerk, eps=eps, precision=prec)
                torch.cuda.synchronize(dev)
                a, j = acc.cpu().numpy(), jerk.cpu().numpy()
                assert np.isfinite(a).all() and np.isfinite(j).all()
                _within(a, j, ra, rj, cond, prec, f"call {call} vs oracle")
                _within(a, j, ctx_a.cpu().numpy(), ctx_j.cpu().numpy(), cond, prec,
                        f"call {call} vs nb_force_jerk_dev")


def test_noalloc_split_blocks_against_oracle(cuda, oracle_mod):
    """n = 5003 with Salpeter masses: a random subset, then every particle
    with no index list; 20 i-blocks over ~300 CTAs, so every i-block is
    split and every output goes through the static array and the fix-up."""
    n, eps = 5003, 1e-3
    m, x, v = ics.plummer(n, 4242, masses=ics.salpeter_masses(n, 4242))
    idx_list = [ics.random_active_subset(n, 1700, 7), np.arange(n, dtype=np.int32)]
    _run_case(cuda, oracle_mod, m, x, v, eps, idx_list, pass_idx=(True, False))


def test_noalloc_whole_blocks_direct_writes(cuda, oracle_mod):
    """n = 1024 (4 j-tiles) with an index list of ~100k entries (repeats
    allowed): 391 i-blocks over at most 341 CTAs, so CTAs cover whole
    i-blocks (direct FP64 writes) next to split ones (fix-up)."""
    n, eps = 1024, 1e-3
    m, x, v = ics.plummer(n, 99, masses=ics.salpeter_masses(n, 99))
    rng = np.random.default_rng(11)
    idx_a = np.tile(rng.permutation(n), 98).astype(np.int32)           # 100,352 entries
    idx_b = rng.integers(0, n, 99_999).astype(np.int32)
    _run_case(cuda, oracle_mod, m, x, v, eps, [idx_a, idx_b])


def test_noalloc_fixup_skipped(cuda, oracle_mod):
    """n = 256 (one j-tile) and 100 i-blocks: one CTA per i-block, every
    result written directly and the fix-up kernel not launched."""
    n, eps = 256, 1e-3
    m, x, v = ics.plummer(n, 5, masses=ics.salpeter_masses(n, 5))
    rng = np.random.default_rng(12)
    idx_a = np.tile(np.arange(n), 100).astype(np.int32)                # 25,600 = 100 blocks
    idx_b = rng.permutation(idx_a).astype(np.int32)
    _run_case(cuda, oracle_mod, m, x, v, eps, [idx_a, idx_b])


def test_noalloc_eps_zero_masked_kernels(cuda, oracle_mod):
    """eps = 0 with distinct particles runs the kernels that zero the
    i == j term; a subset, then every particle."""
    n = 777
    m, x, v = ics.plummer(n, 21)
    idx_list = [ics.random_active_subset(n, 300, 3), np.arange(n, dtype=np.int32)]
    _run_case(cuda, oracle_mod, m, x, v, 0.0, idx_list, pass_idx=(True, False))


def test_noalloc_tiny_eps_takes_masked_kernels(cuda):
    """An eps whose square is below the smallest normal FP32 number is zero
    on the device (subnormals flush to zero); the masked kernels run, and
    the result equals the eps = 0 result bit for bit instead of NaN."""
    torch, _lib, dev = cuda
    n = 600
    m, x, v = ics.plummer(n, 22)
    d_m = torch.from_numpy(m).to(dev)
    d_x = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    d_v = torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    out = {}
    for eps in (0.0, 1e-20):
        for prec in ("ds", "fp32"):
            acc = torch.zeros((n, 3), dtype=torch.float64, device=dev)
            jerk = torch.zeros_like(acc)
            _lib.force_jerk_noalloc(n, d_m, d_x, d_v, None, n, acc, jerk, eps=eps,
                                    precision=prec)
            torch.cuda.synchronize(dev)
            out[eps, prec] = (acc.cpu().numpy(), jerk.cpu().numpy())
    for prec in ("ds", "fp32"):
        a0, j0 = out[0.0, prec]
        a1, j1 = out[1e-20, prec]
        assert np.isfinite(a1).all() and np.isfinite(j1).all()
        assert np.array_equal(a0, a1) and np.array_equal(j0, j1)


def test_noalloc_rejects_bad_sizes(cuda):
    torch, _lib, dev = cuda
    d = torch.zeros(30, dtype=torch.float64, device=dev)
    for n, n_idx in ((0, 1), (10, -1), (10, 11), (2**31, 1)):
        with pytest.raises(_lib.NBodyError) as e:
            _lib.force_jerk_noalloc(n, d, d, d, None, n_idx, d, d, eps=1e-3)
        assert e.value.status == _lib.NB_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        _lib.force_jerk_noalloc(10, d, d, d, None, 1, d, d, eps=1e-3, precision="DS")
