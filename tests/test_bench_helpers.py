"""Host helpers of bench.py (no GPU): the rank correlation used by the
timing-stability report, against its definition and a library routine."""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_spearman_special_cases():
    assert bench.spearman([1, 2, 3, 4], [10, 20, 30, 40]) == pytest.approx(1.0)
    assert bench.spearman([1, 2, 3, 4], [4, 3, 2, 1]) == pytest.approx(-1.0)
    # one adjacent swap of n = 4: 1 - 6 * 2 / (4 * 15)
    assert bench.spearman([1, 2, 3, 4], [1, 3, 2, 4]) == pytest.approx(0.8)


@pytest.mark.parametrize("seed", range(5))
def test_spearman_matches_scipy_with_ties(seed):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 6, 40).astype(float)   # many ties
    b = a + rng.normal(0, 2, 40)
    assert bench.spearman(a, b) == pytest.approx(stats.spearmanr(a, b).statistic, abs=1e-12)


def test_traffic_records_are_well_formed():
    # Every DRAM-traffic record names an existing ncu summary and existing
    # kernel sources; the roofline lookup returns a record's bytes exactly
    # when its source hash matches the current sources.
    import json
    path = os.path.join(ROOT, "profiles", "traffic.json")
    rec = json.load(open(path))
    assert rec["captures"]
    for e in rec["captures"]:
        assert os.path.exists(os.path.join(ROOT, "profiles", e["summary"])), e["summary"]
        assert e["dram_bytes"] > 0 and e["algorithmic_bytes_gemm_kernel"] > 0
        M, N, K = e["shape"]
        assert M > 0 and N > 0 and K > 0
        for f in e["source_files"]:
            assert os.path.exists(os.path.join(ROOT, "paper_2507_15277_gb300", "csrc", f)), f
        current = bench.source_sha256(e["source_files"]) == e["source_sha256"]
        got = bench.traffic_for(e["kernel"], tuple(e["shape"]))
        assert got == (e["dram_bytes"] if current else None)
    assert bench.traffic_for("no_such_kernel", (1, 1, 1)) is None
