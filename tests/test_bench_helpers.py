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


def test_selection_by_kind_on_a_synthetic_table(tmp_path):
    # Three variants of each kind on 8 shapes; the family's per-shape best is
    # a BF16x3 variant on the large shapes and a SIMT one on the small ones.
    pt = pytest.importorskip("paper_2507_15277_gb300")
    vs = pt.variants()
    by_kind = {k: [v["name"] for v in vs if v["kind"] == k][:3] for k in (0, 1, 2)}
    shapes = [(m, n, k) for m in (128, 4096) for n in (128, 4096) for k in (128, 4096)]
    rng = np.random.default_rng(0)
    path = str(tmp_path / "table.csv")
    with open(path, "w") as f:
        f.write("shape_idx,M,N,K,transA,transB,variant,status,valid,median_ms,mean_ms,min_ms,reps,tflops,gbs,max_err\n")
        for s, (m, n, k) in enumerate(shapes):
            big = m * n * k > 128 ** 3 * 64
            for kind, names in by_kind.items():
                for j, name in enumerate(names):
                    t = (1.0 + 0.3 * j + 0.1 * rng.random()) * (2.0 if (kind == 0) == big else 1.0)
                    f.write("%d,%d,%d,%d,N,N,%s,0,1,%.6f,%.6f,%.6f,5,1,1,0\n" % (s, m, n, k, name, t, t, t))
    train, held = list(range(0, 8, 2)), list(range(1, 8, 2))
    res = bench.selection_by_kind(pt, path, train, held, str(tmp_path))
    assert set(res) == {"fp32_simt", "3xtf32", "bf16x3"}
    for label, r in res.items():
        assert r["variants"] == 3
        for k in ("k1", "k2", "k4", "k8"):
            own, fam = r[k]["own_best_pct"], r[k]["family_best_pct"]
            assert 0 < fam <= own <= 100 + 1e-9        # the family's best is at least as fast
        assert r["k4"]["own_best_pct"] == pytest.approx(100.0)   # every variant of the kind chosen
    # neither single kind reaches the family's best on every held-out shape
    assert all(r["k8"]["family_best_pct"] < 100.0 for r in res.values())
