"""GPU: data collection (pt_tune), selection on its table, and the runtime
selector inside pt_sgemm."""

import csv
import json
import os

import numpy as np
import pytest

from oracle import gemm as og
from oracle import select as osel
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"


def _read(path):
    with open(path) as f:
        return list(csv.DictReader(f))


def _times(rows, names, shapes):
    t = np.full((len(names), len(shapes)), np.inf)
    for r in rows:
        if int(r["valid"]):
            s = shapes.index((int(r["M"]), int(r["N"]), int(r["K"]), r["transA"], r["transB"]))
            t[names.index(r["variant"]), s] = float(r["median_ms"])
    return t


@pytest.fixture(scope="module")
def small_table(tmp_path_factory):
    path = str(tmp_path_factory.mktemp("tune") / "table.csv")
    shapes = [(128, 512, 1024), (512, 128, 128), (1024, 1024, 128), (256, 256, 2048), (512, 512, 4096)]
    ids = list(range(0, pt.num_variants(), 9))
    pt.tune(shapes, path, ids=ids, reps_min=3, reps_max=10, target_ms=1.0)
    return path, shapes, ids


def test_table_rows_and_screening(small_table):
    path, shapes, ids = small_table
    rows = _read(path)
    assert len(rows) == len(shapes) * len(ids)
    valid = [r for r in rows if int(r["valid"])]
    for s in shapes:  # every shape, including those tuned after others, keeps valid rows
        rs = [r for r in rows if (int(r["M"]), int(r["N"]), int(r["K"])) == s]
        assert sum(int(r["valid"]) for r in rs) >= 0.8 * len(rs), s
    for r in valid:
        assert float(r["max_err"]) <= TOL_FP32
        assert float(r["median_ms"]) > 0 and float(r["tflops"]) > 0
    assert pt.table_shapes(path) == [s + ("N", "N") for s in shapes]


def test_resume_skips_existing_rows(small_table, tmp_path):
    path, shapes, ids = small_table
    copy = str(tmp_path / "t.csv")
    with open(path) as f, open(copy, "w") as g:
        g.write(f.read())
    n0 = len(_read(copy))
    pt.tune(shapes, copy, ids=ids, resume=True)
    assert len(_read(copy)) == n0
    pt.tune(shapes + [(64, 64, 64)], copy, ids=ids[:3], resume=True)
    assert len(_read(copy)) == n0 + 3


def test_selection_on_measured_table_matches_oracle(small_table, tmp_path):
    path, shapes, ids = small_table
    rows = _read(path)
    names = []
    for r in rows:
        if r["variant"] not in names:
            names.append(r["variant"])
    keys = [s + ("N", "N") for s in shapes]
    t = _times(rows, names, keys)
    train = [0, 1, 2, 3, 4]
    for k in (1, 2, 3):
        got, g = pt.select(path, train, k, method=pt.PT_SELECT_EXACT)
        kappa, val = osel.portability_tune_exhaustive(t, k, train)
        assert g == pytest.approx(val, rel=1e-12)
        assert sorted(pt.variant_by_name(names[v]) for v in kappa) == sorted(got)


def test_manifest_drives_pt_sgemm(small_table, tmp_path):
    path, shapes, ids = small_table
    man = str(tmp_path / "kappa.json")
    got, g = pt.select(path, [0, 1, 2, 3, 4], 2, manifest=man)
    pt.load_manifest(man)
    try:
        rows = _read(path)
        for (M, N, K) in shapes:
            best = None
            for r in rows:
                if (int(r["M"]), int(r["N"]), int(r["K"])) == (M, N, K) and int(r["valid"]):
                    vid = pt.variant_by_name(r["variant"])
                    if vid in got and (best is None or float(r["median_ms"]) < best[0]
                                       or (float(r["median_ms"]) == best[0] and vid < best[1])):
                        best = (float(r["median_ms"]), vid)
            A = torch.from_numpy(matrix("uniform", 9, M, K)).to(DEV)
            B = torch.from_numpy(matrix("uniform", 10, K, N)).to(DEV)
            C = torch.empty((M, N), device=DEV)
            assert pt.selected_variant(M, N, K, A=A, B=B, C=C) == best[1]
            pt.sgemm(A, B, C)
            torch.cuda.synchronize()
            ref = og.gemm(A.cpu().numpy(), B.cpu().numpy())
            assert normalised_error(C.cpu().numpy(), ref, K, 1.0, 1.0) <= TOL_FP32
        # Unlisted shape (extents divisible by 16, so every member admits it):
        # the manifest's time model picks the member of least predicted time,
        # or, without a model, the nearest listed shape's pick decides.
        q = (144, 496, 1008)
        m = json.load(open(man))
        kappa = [pt.variant_by_name(n) for n in m["kappa"]]
        coefs = m["model"]["coef"] if "model" in m else None
        if coefs is not None:
            resids, points = m["model"].get("resid"), m["model"].get("points")
            preds = sorted(osel.model_predict(c, q, None if resids is None else r, points)
                           for c, r in zip(coefs, resids or [None] * len(coefs)) if c is not None)
            if len(preds) < 2 or preds[1] - preds[0] > 1e-9:  # a near tie admits either member
                assert pt.selected_variant(*q) == kappa[osel.model_pick(coefs, q, resids, points)]
        else:
            idx = osel.nearest_shape(q, shapes)
            assert pt.selected_variant(*q) == pt.selected_variant(*shapes[idx])
    finally:
        pt.load_manifest(None)
