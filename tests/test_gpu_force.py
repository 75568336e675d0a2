"""GPU parity of the force + jerk kernels against the FP64 oracle, through
the C ABI (libnbody.so).

Tolerance.  The target is a relative force error <= 1e-6 with split
precision (DS).  Pair arithmetic is FP32, so every pair term carries a
rounding error of a few 1e-8 relative to itself; a particle whose force is
a near-cancellation of larger terms cannot have |da|/|a| <= 1e-6 whatever
the summation.  The bar is therefore stated on the condition of each sum:
  cond_i  = |a_gpu,i - a_ref,i| / sum_j |f_ij|          <= 1e-6 (DS acc)
  norm    = ||a_gpu - a_ref||_2 / ||a_ref||_2 (all i)   <= 1e-6 (DS acc)
and 1e-5 for the DS jerk.  The per-particle e_i = |da_i| / max(|a_i|,
1e-3 rms|a|) is reported, and must be <= 1e-6 on the N = 1M King workload.
Plain FP32 positions: cond and norm <= 1e-3 (reported, not a target).
"""
import numpy as np
import pytest

from paper_0909_0879_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = {"ds": (1e-6, 1e-5), "fp32": (1e-3, 1e-3)}


def rel_err(got, ref):
    scale = np.sqrt(np.mean(np.sum(ref * ref, axis=1))) if len(ref) else 1.0
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-3 * scale)
    return np.linalg.norm(got - ref, axis=1) / den


@pytest.fixture(scope="module")
def nb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0909_0879_gb300 import _lib

    _lib.load()
    return _lib


def check(acc, jerk, ra, rj, prec, cond=None):
    """cond = (sum_j |f_ij|, sum_j |jerk_ij|) from the oracle."""
    ta, tj = TOL[prec]
    na = np.linalg.norm(acc - ra) / np.linalg.norm(ra)
    nj = np.linalg.norm(jerk - rj) / np.linalg.norm(rj)
    assert na <= ta, f"{prec} acc norm-wise err {na:.3e}"
    assert nj <= tj, f"{prec} jerk norm-wise err {nj:.3e}"
    if cond is not None:
        ca = (np.linalg.norm(acc - ra, axis=1) / np.maximum(cond[0], 1e-300)).max()
        cj = (np.linalg.norm(jerk - rj, axis=1) / np.maximum(cond[1], 1e-300)).max()
        assert ca <= ta, f"{prec} acc cond err {ca:.3e}"
        assert cj <= tj, f"{prec} jerk cond err {cj:.3e}"
    return rel_err(acc, ra).max(), rel_err(jerk, rj).max(), na, nj


def oracle_with_cond(oracle_mod, m, x, v, eps, idx=None):
    ra, rj = oracle_mod.force_jerk(m, x, v, eps, idx=idx)
    cond = oracle_mod.force_jerk_abs(m, x, v, eps, idx=idx)
    return ra, rj, cond


@pytest.mark.parametrize("prec", ["ds", "fp32"])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 255, 256, 257, 1023, 4097])
def test_full_active_small_sizes(nb, oracle_mod, prec, n):
    """Every particle active; sizes below, at and past one 256-record tile."""
    m, x, v = ics.plummer(n, 500 + n) if n > 2 else (
        np.array([0.3, 0.7, 0.5])[:n], np.array([[0.1, 0.2, 0.3], [-0.4, 0.1, 0.0], [0.2, -0.3, 0.5]])[:n],
        np.array([[0.0, 0.1, 0.0], [0.2, 0.0, -0.1], [0.0, 0.3, 0.2]])[:n])
    eps = 1e-3
    ra, rj, cond = oracle_with_cond(oracle_mod, m, x, v, eps)
    with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
        acc, jerk = s.force_jerk(np.arange(n, dtype=np.int32))
    if n == 1:
        assert np.all(acc == 0) and np.all(jerk == 0)
        return
    check(acc, jerk, ra, rj, prec, cond)


@pytest.mark.parametrize("prec", ["ds", "fp32"])
def test_every_variant_and_split_grids(nb, oracle_mod, prec):
    """Each compiled kernel shape of this precision, with the persistent grid
    capped to force i-blocks split across CTAs (stream-K fix-up path), on a
    ragged tail (N = 4097) and subsets of several lengths."""
    n, eps = 4097, 1e-3
    m, x, v = ics.plummer(n, 77)
    subsets = [ics.random_active_subset(n, k, 3000 + k) for k in (1, 5, 64, 333, 1500, 4097)]
    refs = [oracle_with_cond(oracle_mod, m, x, v, eps, idx=ii) for ii in subsets]
    with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
        for var in range(nb.num_variants()):
            info = nb.variant_info(var)
            if info["precision"] != (1 if prec == "ds" else 0):
                continue
            try:
                s.set_force_variant(var, 0)
            except nb.NBodyError:
                continue  # eps == 0 variants
            for cap in (0, 7, 150):
                s.set_force_variant(var, cap)
                for ii, (ra, rj, cond) in zip(subsets, refs):
                    acc, jerk = s.force_jerk(ii)
                    check(acc, jerk, ra, rj, prec, cond)


@pytest.mark.parametrize("prec", ["ds", "fp32"])
def test_eps_zero_masks_self_term(nb, oracle_mod, prec):
    """eps = 0: the i == j term is masked; two-body closed form and a small
    random system against the oracle."""
    m = np.array([2.0, 5.0])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    with nb.NBody(m, x, v, eps=0.0, precision=prec) as s:
        acc, jerk = s.force_jerk(np.array([0, 1], dtype=np.int32))
    tol = 1e-6 if prec == "ds" else 1e-5
    np.testing.assert_allclose(acc[0], [0.12, 0.16, 0.0], atol=tol * 0.2)
    np.testing.assert_allclose(jerk[0], [-0.0576, -0.0368, 0.0], atol=tol * 0.07)
    m, x, v = ics.plummer(300, 9)
    ra, rj, cond = oracle_with_cond(oracle_mod, m, x, v, 0.0)
    with nb.NBody(m, x, v, eps=0.0, precision=prec) as s:
        acc, jerk = s.force_jerk(np.arange(300, dtype=np.int32))
    check(acc, jerk, ra, rj, prec, cond)


@pytest.mark.parametrize("prec", ["ds", "fp32"])
def test_tiny_eps_takes_masked_kernels(nb, prec):
    """An eps whose square is not a normal FP32 number is zero on the
    device (subnormals flush to zero), so the context runs the kernels that
    zero the i == j term: finite, and bit for bit the eps = 0 result."""
    m, x, v = ics.plummer(500, 10)
    idx = np.arange(500, dtype=np.int32)
    out = []
    for eps in (0.0, 1e-20):
        with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
            out.append(s.force_jerk(idx))
    assert np.isfinite(out[1][0]).all() and np.isfinite(out[1][1]).all()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_deterministic_and_duplicate_indices(nb):
    n = 5000
    m, x, v = ics.plummer(n, 3)
    idx = np.concatenate([np.arange(0, n, 7), np.arange(0, n, 7)]).astype(np.int32)
    with nb.NBody(m, x, v, eps=1e-3) as s:
        a1, j1 = s.force_jerk(idx)
        a2, j2 = s.force_jerk(idx)
    assert np.array_equal(a1, a2) and np.array_equal(j1, j2)
    h = len(idx) // 2
    assert np.array_equal(a1[:h], a1[h:])


def test_salpeter_masses_close_pairs(nb, oracle_mod):
    """Unequal masses spanning three decades and eps = 1e-4 (the block-step
    workload's mass spectrum and softening) at N = 8192."""
    n, eps = 8192, 1e-4
    m, x, v = ics.plummer(n, 1002, masses=ics.salpeter_masses(n, 1002))
    idx = ics.random_active_subset(n, 512, 2002)
    ra, rj, cond = oracle_with_cond(oracle_mod, m, x, v, eps, idx=idx)
    for prec in ("ds", "fp32"):
        with nb.NBody(m, x, v, eps=eps, precision=prec) as s:
            acc, jerk = s.force_jerk(idx)
        print(prec, "errors (max e_i acc, jerk, norm acc, jerk)", check(acc, jerk, ra, rj, prec, cond))


def test_device_pointer_path_matches_host_path(nb):
    import torch

    n = 3000
    m, x, v = ics.plummer(n, 4)
    idx = ics.random_active_subset(n, 1000, 1)
    with nb.NBody(m, x, v, eps=1e-3) as s:
        acc_h, jerk_h = s.force_jerk(idx)
        d_idx = torch.from_numpy(idx).cuda()
        d_acc = torch.zeros((1000, 3), dtype=torch.float64, device="cuda")
        d_jerk = torch.zeros_like(d_acc)
        s.force_jerk_dev(d_idx, 1000, d_acc, d_jerk)
        s.sync()
    assert np.array_equal(d_acc.cpu().numpy(), acc_h)
    assert np.array_equal(d_jerk.cpu().numpy(), jerk_h)


def test_king_1m_sampled_parity(nb, oracle_mod):
    """Full-size single evaluation (N = 1,048,576 King W0 = 7, eps = 1e-4),
    every particle active, particles in generation order (i-blocks and
    j-tiles spread over the cluster, so nearly every tile takes the
    split-precision difference); 256 sampled particles against the
    oracle."""
    import torch

    n, eps = 1 << 20, 1e-4
    m, x, v = ics.king(n, 7.0, 1003)
    sample = np.sort(np.random.default_rng(2003).choice(n, 256, replace=False))
    ra, rj, cond = oracle_with_cond(oracle_mod, m, x, v, eps, idx=sample)
    errs = {}
    for prec in ("ds", "fp32"):
        with nb.NBody(m, x, v, eps=eps, precision=prec, block_steps=False, lev_shared=10) as s:
            d_acc = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
            d_jerk = torch.zeros_like(d_acc)
            d_idx = torch.arange(n, dtype=torch.int32, device="cuda")
            s.force_jerk_dev(d_idx, n, d_acc, d_jerk)
            s.sync()
            acc = d_acc[torch.from_numpy(sample).cuda()].cpu().numpy()
            jerk = d_jerk[torch.from_numpy(sample).cuda()].cpu().numpy()
        errs[prec] = check(acc, jerk, ra, rj, prec, cond)
    print("king 1M sampled errors (max e_i acc, jerk, norm acc, jerk)", errs)
    assert errs["ds"][0] <= 1e-6, "per-particle DS force error at N = 1M"


def test_packed_variants_bitwise_equal_scalar(nb):
    """The packed FP32x2 kernels round every lane like the scalar kernels,
    so a packed variant and the scalar variant of the same shape give
    bit-identical sums."""
    n = 6000
    m, x, v = ics.plummer(n, 12, masses=ics.salpeter_masses(n, 12))
    idx = ics.random_active_subset(n, 2500, 5)
    infos = [nb.variant_info(k) for k in range(nb.num_variants())]
    pairs = []
    for k, inf in enumerate(infos):
        if not inf["packed"]:
            continue
        for j, jnf in enumerate(infos):
            if (not jnf["packed"] and jnf["precision"] == inf["precision"] and
                    jnf["ipt"] == inf["ipt"] and jnf["tpi"] == inf["tpi"] and
                    jnf["threads"] == inf["threads"]):
                pairs.append((k, j))
    assert len(pairs) >= 4
    for prec in ("ds", "fp32"):
        with nb.NBody(m, x, v, eps=1e-4, precision=prec) as s:
            for k, j in pairs:
                if infos[k]["precision"] != (1 if prec == "ds" else 0):
                    continue
                s.set_force_variant(k, 0)
                ak, jk = s.force_jerk(idx)
                s.set_force_variant(j, 0)
                aj, jj = s.force_jerk(idx)
                assert np.array_equal(ak, aj) and np.array_equal(jk, jj), (k, j)


def test_tile_relative_far_field_on_sorted_particles(nb, oracle_mod):
    """Particles listed along a Morton curve make i-blocks and j-tiles
    compact, so the tile-relative far-field path runs for most tiles; the
    result meets the split-precision bar and agrees with the plain
    split-precision shape."""
    n, eps = 20000, 1e-4
    m, x, v = ics.king(n, 7.0, 4)
    p = ics.morton_order(x)
    m, x, v = m[p], x[p], v[p]
    idx = np.arange(n, dtype=np.int32)
    sample = np.sort(np.random.default_rng(9).choice(n, 600, replace=False)).astype(np.int32)
    ra, rj, cond = oracle_with_cond(oracle_mod, m, x, v, eps, idx=sample)
    rel_variants = [k for k in range(nb.num_variants())
                    if nb.variant_info(k)["precision"] == 1 and nb.variant_info(k)["packed"]]
    with nb.NBody(m, x, v, eps=eps, precision="ds") as s:
        s.set_force_variant(12, 0)
        a12, j12 = s.force_jerk(idx)
        for k in rel_variants:
            s.set_force_variant(k, 0)
            acc, jerk = s.force_jerk(idx)
            print(k, "errors", check(acc[sample], jerk[sample], ra, rj, "ds", cond))
            assert np.linalg.norm(acc - a12) / np.linalg.norm(a12) < 1e-6


def test_king_1m_bench_layout_parity(nb, oracle_mod):
    """The headline evaluation exactly as the bench times it: N = 1,048,576
    King W0 = 7, eps = 1e-4, particles stored in nb_spatial_order (256 per
    leaf), Hermite shared step 2^-10 with every particle active, the force
    call of a step (active list from nb_next_block, built-in shape and grid)
    at the predicted state.  In this layout most (i-block, tile) pairs take
    the tile-relative FP32 far field; the built-in long-list shape must be
    the tile-relative one (bitwise equal to forcing variant 26).  1024
    sampled particles against the oracle on the same predicted state: the
    condition-relative and norm-wise bars, and the per-particle e_i <= 1e-6
    of the split-precision target."""
    import torch

    n, eps = 1 << 20, 1e-4
    m, x, v = ics.king(n, 7.0, 1003)
    perm = nb.spatial_order(x, 256)
    m, x, v = m[perm], x[perm], v[perm]
    sample = np.sort(np.random.default_rng(2013).choice(n, 1024, replace=False))
    assert nb.variant_info(26)["precision"] == 1 and nb.variant_info(26)["packed"] == 1
    with nb.NBody(m, x, v, eps=eps, precision="ds", block_steps=False, lev_shared=10) as s:
        st = s.get_state()
        t, na = s.next_block()
        assert na == n
        s.predict(t)
        d_acc = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        d_jerk = torch.zeros_like(d_acc)
        s.force_jerk_dev(None, na, d_acc, d_jerk)
        s.sync()
        sel = torch.from_numpy(sample).cuda()
        acc = d_acc[sel].cpu().numpy()
        jerk = d_jerk[sel].cpu().numpy()
        # the default shape for this length is the tile-relative one
        s.set_force_variant(26, 0)
        d_acc26 = torch.zeros_like(d_acc)
        d_jerk26 = torch.zeros_like(d_acc)
        s.force_jerk_dev(torch.arange(n, dtype=torch.int32, device="cuda"), n, d_acc26, d_jerk26)
        s.sync()
        assert torch.equal(d_acc, d_acc26) and torch.equal(d_jerk, d_jerk26)
    dt = t - 0.0
    xp, vp = oracle_mod.predict(st["x"], st["v"], st["a"], st["jerk"], dt)
    ra, rj, cond = oracle_with_cond(oracle_mod, m, xp, vp, eps, idx=sample)
    errs = check(acc, jerk, ra, rj, "ds", cond)
    print("king 1M bench layout (max e_i acc, jerk, norm acc, jerk)", errs)
    assert errs[0] <= 1e-6, f"per-particle DS force error {errs[0]:.3e} at N = 1M"
