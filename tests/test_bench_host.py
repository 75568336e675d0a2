"""Host-side helpers of bench.py (no GPU): the force-error summary against
the oracle that the bench line reports, and the lookup of the committed
DRAM-traffic record."""
import hashlib
import json
import os

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_force_error_summary_matches_its_definitions():
    rng = np.random.default_rng(3)
    ra = rng.normal(size=(200, 3))
    rj = rng.normal(size=(200, 3))
    # known per-row errors: row k is off by (k + 1) * 1e-9 along x
    da = np.zeros_like(ra)
    da[:, 0] = (np.arange(200) + 1) * 1e-9
    dj = 2.0 * da
    cond = (np.full(50, 4.0), np.full(50, 8.0))
    out = bench.force_error(ra + da, rj + dj, ra, rj, cond)
    rms = np.sqrt(np.mean(np.sum(ra * ra, 1)))
    ei = np.abs(da[:, 0]) / np.maximum(np.linalg.norm(ra, axis=1), 1e-3 * rms)
    assert np.isclose(out["acc_max_ei"], ei.max())
    assert np.isclose(out["acc_p99_ei"], np.quantile(ei, 0.99))
    assert np.isclose(out["acc_norm"], np.linalg.norm(da) / np.linalg.norm(ra))
    assert np.isclose(out["jerk_norm"], np.linalg.norm(dj) / np.linalg.norm(rj))
    # condition-relative errors use the first len(cond) rows only
    assert np.isclose(out["acc_cond_max"], (50 * 1e-9) / 4.0)
    assert np.isclose(out["jerk_cond_max"], (2 * 50 * 1e-9) / 8.0)
    exact = bench.force_error(ra, rj, ra, rj)
    assert exact["acc_max_ei"] == 0.0 and "acc_cond_max" not in exact


def test_traffic_record_belongs_to_the_kernel_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "force_jerk_ds_traffic.json")))
    src = os.path.join(ROOT, "paper_0909_0879_gb300", "csrc", "nb_force.cu")
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    got = bench.force_traffic_from_profile(rec["n"])
    if cur == rec["source_sha256"]:
        assert got == rec["dram_bytes_per_launch"]
        # traffic above the algorithmic bytes: re-reads of j-tiles through L2
        assert rec["dram_bytes_per_launch"] >= rec["algorithmic_bytes_per_launch"]
    else:
        assert got is None
    assert bench.force_traffic_from_profile(rec["n"] + 1) is None
