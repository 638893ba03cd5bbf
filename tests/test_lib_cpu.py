"""Host-side library checks (no GPU): the C ABI loads and exports every
declared symbol, the registry follows the variant-space rules, and the C++
selector / scorer / manifest agree with the oracle on synthetic tables."""

import json
import math
import os
import re

import numpy as np
import pytest

from oracle import select as osel

pt = pytest.importorskip("paper_2507_15277_gb300")
from paper_2507_15277_gb300 import _lib  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pt_sgemm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _lib.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES), "binding and header disagree"


def test_registry_rules():
    n = pt.num_variants()
    assert 300 <= n <= 456  # the GPU parity tests cover ids 0..455
    names = set()
    simt = []
    for i in range(n):
        d = pt.variant(i)
        assert d["id"] == i
        assert d["name"] not in names
        names.add(d["name"])
        assert pt.variant_by_name(d["name"]) == i
        assert d["smem_bytes"] <= 232448
        if d["kind"] != 0:
            # split-precision tensor-core variants: 128-row tiles (256 for a CTA pair), TMA, any layout
            assert d["kind"] in (1, 2, 3) and d["bn"] in (32, 64, 128, 256)
            assert d["bm"] == (256 if "_2sm" in d["name"] else 128)
            assert d["name"].startswith({1: "tc3xtf32_", 2: "tcbf16x3_", 3: "tc3xf16_"}[d["kind"]])
            # fused versions read B (or A) themselves: transB (transA) = 'N' only; the others take any layout
            assert d["loader"] == 1 and d["trans_mask"] == (1 if "_fab" in d["name"] else 5 if "_fb" in d["name"]
                                                            else 3 if "_fa" in d["name"] else 15)
            # epilogue + producer + MMA warps (+ four converter warps when B is split in the kernel)
            fused = "_fb" in d["name"] or "_fa" in d["name"]
            conv = (2 if d["bn"] >= 128 else 4) if fused else 0  # converter warps
            assert d["threads"] == 32 * (4 * max(1, d["bn"] // 128) + 2 + conv)
            want = (pt.PT_SCHED_STREAMK if d["name"].endswith("_stk") else
                    pt.PT_SCHED_TILE if d["splitk"] > 1 else pt.PT_SCHED_PERSISTENT)
            assert d["schedule"] == want
            row = d["bk"] * (4 if d["kind"] == 1 else 2)  # one swizzle row: 128, 64 or 32 bytes
            assert row == (64 if "_sw64" in d["name"] else 32 if "_sw32" in d["name"] else 128)
            continue
        simt.append(i)
        assert d["schedule"] == pt.PT_SCHED_TILE
        assert d["bm"] % d["wm"] == 0 and d["bn"] % d["wn"] == 0
        assert (d["wm"] // d["tm"]) * (d["wn"] // d["tn"]) * d["kl"] == 32
        assert d["threads"] == 32 * (d["bm"] // d["wm"]) * (d["bn"] // d["wn"])
        assert d["threads"] in (64, 128, 256, 512)
        assert d["bk"] % (4 * d["kl"]) == 0
        assert d["smem_bytes"] <= 232448
        assert d["bm"] % d["splitk"] == 0
        assert d["tm"] * d["tn"] <= 64
    assert {pt.variant(i)["kind"] for i in range(n)} == {0, 1, 2, 3}
    assert all(pt.variant(i)["kind"] == 0 for i in range(len(simt)))  # SIMT family first
    d0 = pt.variant(pt.default_variant())
    assert (d0["bm"], d0["bn"], d0["bk"], d0["vec"], d0["loader"], d0["trans_mask"]) == (128, 128, 8, 1, 0, 15)
    for key, values in (("splitk", {1, 2, 4, 8}), ("loader", {0, 1}), ("vec", {1, 2, 4}),
                        ("stages", {2, 3, 4}), ("bk", {8, 16, 32}), ("kl", {1, 2, 4}), ("fma2", {0, 1})):
        assert {pt.variant(i)[key] for i in simt} == values, key


def test_argument_validation_without_gpu():
    lib = _lib.lib()
    rc = lib.pt_sgemm(b"X", b"N", 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None)
    assert rc == _lib.PT_EINVAL and lib.pt_last_error_arg() == 1
    rc = lib.pt_sgemm(b"N", b"N", -1, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None)
    assert rc == _lib.PT_EINVAL and lib.pt_last_error_arg() == 3
    rc = lib.pt_sgemm(b"N", b"N", 4, 4, 8, 1.0, None, 7, None, 4, 0.0, None, 4, None)
    assert rc == _lib.PT_EINVAL and lib.pt_last_error_arg() == 8
    rc = lib.pt_sgemm(b"N", b"T", 4, 4, 8, 1.0, None, 8, None, 4, 0.0, None, 4, None)
    assert rc == _lib.PT_EINVAL and lib.pt_last_error_arg() == 10
    rc = lib.pt_sgemm(b"N", b"N", 4, 5, 8, 1.0, None, 8, None, 5, 0.0, None, 4, None)
    assert rc == _lib.PT_EINVAL and lib.pt_last_error_arg() == 13
    # Empty output: nothing to do, no device touched.
    assert lib.pt_sgemm(b"N", b"N", 0, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None) == 0
    assert lib.pt_variant_desc(10 ** 6, None) == _lib.PT_EINVAL
    assert lib.pt_variant_by_name(b"no_such_variant") == _lib.PT_EINVAL


def test_failure_hooks_arguments_without_gpu():
    lib = _lib.lib()
    o = _lib.TuneOpts()
    o.fail_launch = 77
    lib.pt_tune_default_opts(o)
    assert o.fail_launch == 0 and o.warmup == 2 and o.tol == 2e-6
    assert lib.pt_debug_streamk_wait(3 * 10 ** 9, 0) == _lib.PT_EINVAL and lib.pt_last_error_arg() == 1
    assert lib.pt_debug_streamk_wait(1000, 2) == _lib.PT_EINVAL and lib.pt_last_error_arg() == 2
    assert lib.pt_debug_streamk_wait(1000, 1) == 0
    assert lib.pt_debug_streamk_wait(0, 0) == 0      # back to normal operation
    # a negative launch index is refused before any device work
    o.fail_launch = -1
    shapes = (_lib.Shape * 1)(_lib.Shape(8, 8, 8, b"N", b"N"))
    assert lib.pt_tune(shapes, 1, None, 0, o, b"/nonexistent/t.csv") == _lib.PT_EINVAL


# ---- selection against the oracle ------------------------------------------------------

HEADER_CSV = "shape_idx,M,N,K,transA,transB,variant,status,valid,median_ms,mean_ms,min_ms,reps,tflops,gbs,max_err"


def write_table(path, times, shapes=None, names=None):
    V, S = times.shape
    names = names or [pt.variant(i)["name"] for i in range(V)]
    shapes = shapes or [(64 * (s + 1), 128, 256, "N", "N") for s in range(S)]
    with open(path, "w") as f:
        f.write(HEADER_CSV + "\n")
        for s in range(S):
            for v in range(V):
                t = times[v, s]
                ok = np.isfinite(t)
                m, n, k, ta, tb = shapes[s]
                f.write("%d,%d,%d,%d,%s,%s,%s,%d,%d,%.17g,%.17g,%.17g,5,1,1,0\n" % (
                    s, m, n, k, ta, tb, names[v], 0 if ok else -2, int(ok), t if ok else 0.0,
                    t if ok else 0.0, t if ok else 0.0))
    return names, shapes


def random_table(seed, V, S, invalid=0.1):
    rng = np.random.default_rng(seed)
    t = np.exp(rng.normal(0, 0.6, size=(V, S)))
    t[rng.random((V, S)) < invalid] = np.inf
    for s in range(S):
        if not np.isfinite(t[:, s]).any():
            t[0, s] = 1.0
    return t


def test_golden_tiny_table(tmp_path):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "select_tiny.json")))
    t = np.array(g["times"])
    path = str(tmp_path / "t.csv")
    write_table(path, t)
    for k, opt in g["optimum"].items():
        ids, val = pt.select(path, [0, 1, 2], int(k), method=pt.PT_SELECT_EXACT)
        assert ids == opt["kappa"] and val == pytest.approx(opt["value"], rel=1e-12)
        ids2, val2 = pt.select(path, [0, 1, 2], int(k), method=pt.PT_SELECT_GREEDY_SWAP)
        assert val2 == pytest.approx(opt["value"], rel=1e-12), "swap search escapes the greedy trap"


@pytest.mark.parametrize("seed", range(8))
def test_exact_selection_matches_oracle(seed, tmp_path):
    t = random_table(seed, 9, 7)
    path = str(tmp_path / "t.csv")
    write_table(path, t)
    train = [0, 2, 3, 5, 6] if seed % 2 else list(range(7))
    for k in (1, 2, 3, 4):
        ids, val = pt.select(path, train, k, method=pt.PT_SELECT_EXACT)
        kappa, oval = osel.portability_tune_exhaustive(t, k, train)
        assert val == pytest.approx(oval, rel=1e-12)
        assert osel.set_performance(t, ids, train) == pytest.approx(oval, rel=1e-12)
        assert ids == kappa


@pytest.mark.parametrize("seed", range(6))
def test_greedy_swap_quality(seed, tmp_path):
    t = random_table(100 + seed, 14, 10, invalid=0.0)
    path = str(tmp_path / "t.csv")
    write_table(path, t)
    S = list(range(10))
    for k in (2, 3, 4):
        _, opt = osel.portability_tune_exhaustive(t, k, S)
        ids, val = pt.select(path, S, k, method=pt.PT_SELECT_GREEDY_SWAP, seed=seed)
        assert len(ids) == k
        assert osel.set_performance(t, ids, S) == pytest.approx(val, rel=1e-12)
        # facility-location bound on the shifted objective, and in practice near-optimal
        lg = np.log(t.min(axis=0)[None, :] / t)
        c = -lg.min()
        f = lambda kap: float(np.sum(np.max(lg[list(kap)] + c, axis=0)))
        kap_opt, _ = osel.portability_tune_exhaustive(t, k, S)
        assert f(ids) >= (1 - 1 / math.e) * f(kap_opt) - 1e-9
        assert val >= 0.97 * opt


def test_score_best_of_set_and_selector(tmp_path):
    t = random_table(7, 8, 12)
    shapes = [(2 ** (6 + s % 4), 2 ** (6 + (s // 4) % 3), 2 ** (7 + s % 3), "N", "N") for s in range(12)]
    shapes = list(dict.fromkeys(shapes))
    t = t[:, :len(shapes)]
    path = str(tmp_path / "t.csv")
    names, _ = write_table(path, t, shapes=shapes)
    S = len(shapes)
    train = list(range(0, S, 2))
    held = list(range(1, S, 2))
    man = str(tmp_path / "m.json")
    ids, val = pt.select(path, train, 3, method=pt.PT_SELECT_EXACT, manifest=man)
    # best-of-set scoring == Eq. 1 on the held-out shapes
    assert pt.score(path, held, ids) == pytest.approx(osel.set_performance(t, ids, held), rel=1e-12)
    # selector-realised: each held-out shape takes the member with the smallest
    # time predicted by the manifest's model (fitted on the training shapes,
    # corrected by the distance-weighted residuals there)
    m = json.load(open(man))
    assert [e["variant"] for e in m["map"]] == [names[osel.best_in_set(t, ids, s)] for s in train]
    tb = osel.per_shape_best(t)
    logs = []
    points = [shapes[s][:3] for s in train]
    coefs = [osel.model_fit(t[v, train], points) for v in ids]
    resids = [osel.model_residuals(c, t[v, train], points) for c, v in zip(coefs, ids)]
    for s in held:
        v = ids[osel.model_pick(coefs, shapes[s][:3], resids, points)]
        tv = t[v, s]
        if not np.isfinite(tv):
            fall = [t[i, s] for i in ids if np.isfinite(t[i, s])]
            tv = fall[0] if fall else t[0, s]
        logs.append(math.log(tb[s] / tv))
    want = math.exp(sum(logs) / len(logs))
    got = pt.score(path, held, mode=pt.PT_SCORE_SELECTOR, manifest=man)
    assert got == pytest.approx(want, rel=1e-12)


def test_manifest_round_trip_and_errors(tmp_path):
    t = random_table(3, 5, 4, invalid=0.0)
    path = str(tmp_path / "t.csv")
    write_table(path, t)
    man = str(tmp_path / "m.json")
    pt.select(path, [0, 1, 2, 3], 2, manifest=man)
    pt.load_manifest(man)
    pt.load_manifest(None)
    bad = str(tmp_path / "bad.json")
    open(bad, "w").write('{"format": "pt-manifest-1", "kappa": ["nope"]}')
    with pytest.raises(pt.PtError) as e:
        pt.load_manifest(bad)
    assert e.value.code == _lib.PT_EFORMAT
    open(bad, "w").write("{not json")
    with pytest.raises(pt.PtError) as e:
        pt.load_manifest(bad)
    assert e.value.code == _lib.PT_EFORMAT
    with pytest.raises(pt.PtError) as e:
        pt.load_manifest(str(tmp_path / "missing.json"))
    assert e.value.code == _lib.PT_EIO


def test_malformed_and_truncated_tables(tmp_path):
    t = random_table(4, 4, 3, invalid=0.0)
    path = str(tmp_path / "t.csv")
    write_table(path, t)
    lines = open(path).read().splitlines()
    trunc = str(tmp_path / "trunc.csv")
    open(trunc, "w").write("\n".join(lines[:-1]) + "\n" + lines[-1][:20] + "\n")
    with pytest.raises(pt.PtError) as e:
        pt.select(trunc, [0], 1)
    assert e.value.code == _lib.PT_EFORMAT
    hdr = str(tmp_path / "hdr.csv")
    open(hdr, "w").write("a,b,c\n")
    with pytest.raises(pt.PtError) as e:
        pt.select(hdr, [0], 1)
    assert e.value.code == _lib.PT_EFORMAT
    # A later row for the same (shape, variant) replaces the earlier one (resume).
    dup = str(tmp_path / "dup.csv")
    name0 = pt.variant(0)["name"]
    open(dup, "w").write("\n".join(lines) + "\n" + "0,64,128,256,N,N,%s,0,1,1e-9,1e-9,1e-9,5,1,1,0\n" % name0)
    ids, val = pt.select(dup, [0], 1)
    assert ids == [0]


def test_table_shape_listing(tmp_path):
    t = random_table(5, 3, 4, invalid=0.0)
    path = str(tmp_path / "t.csv")
    _, shapes = write_table(path, t)
    assert pt.table_shapes(path) == shapes


# ---- k-means and regression-tree selection (Section IV-C) against the oracle ----------

def _sweep_like(seed, V, invalid=0.1):
    sizes = (128, 512, 1024, 4096)
    shapes = [(m, n, k, "N", "N") for m in sizes for n in sizes for k in sizes[:2]]
    return random_table(seed, V, len(shapes), invalid=invalid), shapes


@pytest.mark.parametrize("seed", range(5))
def test_kmeans_selection_matches_oracle(seed, tmp_path):
    t, shapes = _sweep_like(500 + seed, 12)
    path = str(tmp_path / "t.csv")
    write_table(path, t, shapes=shapes)
    train = list(range(0, len(shapes), 2))
    for k in (1, 2, 3, 5):
        ids, val = pt.select(path, train, k, method=pt.PT_SELECT_KMEANS, seed=seed)
        want, _ = osel.kmeans_select(t, k, train, seed=seed)
        assert ids == want, (k, ids, want)
        assert val == pytest.approx(osel.set_performance(t, want, train), rel=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_tree_selection_matches_oracle(seed, tmp_path):
    t, shapes = _sweep_like(600 + seed, 10)
    path = str(tmp_path / "t.csv")
    write_table(path, t, shapes=shapes)
    train = list(range(len(shapes)))
    feats = [tuple(math.log2(x) for x in sh[:3]) for sh in shapes]
    for k in (1, 2, 4, 6):
        ids, val = pt.select(path, train, k, method=pt.PT_SELECT_TREE)
        want, _ = osel.tree_select(t, k, train, feats)
        assert ids == want, (k, ids, want)


def test_tree_manifest_is_the_runtime_selector_for_unlisted_shapes(tmp_path):
    t, shapes = _sweep_like(700, 8, invalid=0.0)
    path = str(tmp_path / "t.csv")
    write_table(path, t, shapes=shapes)
    man = str(tmp_path / "tree.json")
    train = list(range(0, len(shapes), 2))
    pt.select(path, train, 4, method=pt.PT_SELECT_TREE, manifest=man)
    m = json.load(open(man))
    assert m["method"] == "tree" and len(m["tree"]) >= 1

    def descend(q):
        f = [math.log2(x) for x in q]
        node = 0
        while "variant" not in m["tree"][node]:
            nd = m["tree"][node]
            node = nd["left"] if f[nd["feature"]] <= nd["threshold"] else nd["right"]
        return pt.variant_by_name(m["tree"][node]["variant"])

    pt.load_manifest(man)
    try:
        for q in [(200, 300, 700), (2048, 96, 4000), (4096, 4096, 4096), (130, 5000, 129)]:
            assert pt.selected_variant(*q) == descend(q)
        # Listed (training) shapes keep their fastest member.
        s = train[3]
        assert pt.selected_variant(*shapes[s][:3]) == osel.best_in_set(t, [pt.variant_by_name(x) for x in m["kappa"]], s)
    finally:
        pt.load_manifest(None)


def test_kernel_timer_without_launches():
    # No launch in between: nothing recorded, no CUDA call needed.
    pt.kernel_timer_start()
    assert pt.kernel_timer_stop() == (0.0, 0)
    # Stopping a timer that is not running is harmless too.
    assert pt.kernel_timer_stop() == (0.0, 0)


@pytest.mark.parametrize("seed", range(6))
def test_time_model_matches_oracle(seed, tmp_path):
    # Tables on a 4 x 4 x 4 grid of shapes; the manifest's model coefficients
    # equal the oracle's fit, and unlisted shapes get the oracle's pick.
    levels = (128, 512, 1024, 4096)
    shapes = [(m, n, k, "N", "N") for m in levels for n in levels for k in levels]
    t = random_table(100 + seed, 10, len(shapes), invalid=0.15)
    path = str(tmp_path / "t.csv")
    write_table(path, t, shapes=shapes)
    rng = np.random.default_rng(seed)
    train = sorted(rng.choice(len(shapes), 32, replace=False).tolist())
    man = str(tmp_path / "m.json")
    ids, _ = pt.select(path, train, 4, manifest=man)
    ids = [i for i in ids if i >= 0]
    m = json.load(open(man))
    points = [shapes[s][:3] for s in train]
    coefs = [osel.model_fit(t[v, train], points) for v in ids]
    resids = [osel.model_residuals(c, t[v, train], points) for c, v in zip(coefs, ids)]
    for got, want in zip(m["model"]["coef"], coefs):
        if want is None:
            assert got is None
        else:
            assert np.allclose(got, want, rtol=1e-8, atol=1e-8)
    assert [tuple(p) for p in m["model"]["points"]] == [tuple(p) for p in points]
    for got, want in zip(m["model"]["resid"], resids):
        if want is None:
            assert got is None
            continue
        assert [g is None for g in got] == [w is None for w in want]
        assert np.allclose([g for g in got if g is not None], [w for w in want if w is not None], atol=1e-8)
    pt.load_manifest(man)
    try:
        # extents divisible by 16, so that every variant's alignment rules admit them
        for q in [(208, 704, 3008), (128, 4096, 304), (3008, 160, 160), (784, 784, 784), (112, 112, 5008)]:
            preds = sorted(osel.model_predict(c, q, r, points) for c, r in zip(coefs, resids) if c is not None)
            if len(preds) > 1 and preds[1] - preds[0] < 1e-9:
                continue  # a near tie: either member is a correct pick
            assert pt.selected_variant(*q) == ids[osel.model_pick(coefs, q, resids, points)]
        # listed shapes keep their fastest member
        s = train[5]
        assert pt.selected_variant(*shapes[s][:3]) == osel.best_in_set(t, ids, s)
    finally:
        pt.load_manifest(None)


def test_manifest_without_model_uses_nearest_shape(tmp_path):
    # Training shapes with mixed transposes get no model: the nearest listed shape decides.
    shapes = [(128, 128, 128, "N", "N"), (4096, 4096, 4096, "N", "N"), (128, 128, 128, "N", "T"),
              (4096, 4096, 4096, "N", "T")]
    t = np.array([[1.0, 9.0, 1.0, 9.0], [9.0, 1.0, 9.0, 1.0], [5.0, 5.0, 5.0, 5.0]])
    path = str(tmp_path / "t.csv")
    write_table(path, t, shapes=shapes)
    man = str(tmp_path / "m.json")
    ids, _ = pt.select(path, [0, 1, 2, 3], 2, manifest=man)
    assert "model" not in json.load(open(man))
    pt.load_manifest(man)
    try:
        assert pt.selected_variant(200, 200, 200) == 0
        assert pt.selected_variant(3000, 3000, 3000, transB="T") == 1
    finally:
        pt.load_manifest(None)


def test_malformed_time_model_is_rejected(tmp_path):
    # Planted mistakes in the manifest's model block: each must fail to load
    # with PT_EFORMAT; a member without a model, or a model without residuals,
    # loads.
    levels = (128, 512, 1024, 4096)
    shapes = [(m, n, k, "N", "N") for m in levels for n in levels for k in levels]
    t = random_table(7, 6, len(shapes), invalid=0.0)
    path = str(tmp_path / "t.csv")
    write_table(path, t, shapes=shapes)
    man = str(tmp_path / "m.json")
    ids, _ = pt.select(path, list(range(0, 64, 2)), 3, manifest=man)
    good = json.load(open(man))
    assert len(good["model"]["coef"]) == len(good["kappa"])

    def mutated(fn):
        m = json.loads(json.dumps(good))
        fn(m["model"])
        p = str(tmp_path / "bad.json")
        with open(p, "w") as f:
            f.write(json.dumps(m).replace("Infinity", "1e999"))
        return p

    bad = [
        lambda md: md["coef"].pop(),                      # one row fewer than kappa
        lambda md: md["coef"][0].pop(),                   # nine coefficients
        lambda md: md["coef"][0].__setitem__(3, "x"),     # not a number
        lambda md: md["coef"][0].__setitem__(0, float("inf")),  # not finite
        lambda md: md.__setitem__("transA", "NN"),        # not one character
        lambda md: md.pop("transB"),                      # missing field
        lambda md: md["coef"].__setitem__(1, 3.0),        # row neither a list nor null
        lambda md: md["resid"].pop(),                     # one residual row fewer than kappa
        lambda md: md["resid"][0].pop(),                  # a row shorter than the point list
        lambda md: md["resid"][0].__setitem__(2, "x"),    # not a number
        lambda md: md["points"][0].pop(),                 # a point without K
        lambda md: md["points"].__setitem__(1, [0, 512, 512]),  # a point with M = 0
        lambda md: md.pop("points"),                      # residuals without their points
        lambda md: md["coef"].__setitem__(0, None),       # residuals for a member without a model
    ]
    for fn in bad:
        with pytest.raises(pt.PtError) as e:
            pt.load_manifest(mutated(fn))
        assert e.value.code == _lib.PT_EFORMAT
    # A member without a model (null coefficient and residual rows) is
    # allowed, and so is a model without residuals.
    ok = mutated(lambda md: (md["coef"].__setitem__(0, None), md["resid"].__setitem__(0, None)))
    pt.load_manifest(mutated(lambda md: (md.pop("points"), md.pop("resid"))))
    pt.load_manifest(ok)
    try:
        assert pt.selected_variant(208, 704, 3008) in ids
    finally:
        pt.load_manifest(None)


def test_residuals_decide_between_equal_models(tmp_path):
    # Two members with identical models; member 1 runs 0.3 faster than its
    # model at the training shape next to the query and 0.3 slower at the far
    # one, so the library must pick it (without residuals: a tie, member 0).
    simt = [pt.variant(i)["name"] for i in range(pt.num_variants())
            if pt.variant(i)["kind"] == 0 and pt.variant(i)["trans_mask"] == 15 and pt.variant(i)["vec"] == 1][:2]
    zero = [0.0] * 10
    man = {"format": "pt-manifest-1", "kappa": simt,
           "map": [{"m": 4096, "n": 4096, "k": 128, "transA": "N", "transB": "N", "variant": simt[0]}],
           "model": {"transA": "N", "transB": "N", "coef": [zero, zero],
                     "points": [[512, 512, 1024], [4096, 4096, 128]], "resid": [[0.0, 0.0], [-0.3, 0.3]]}}
    path = str(tmp_path / "m.json")
    json.dump(man, open(path, "w"))
    pt.load_manifest(path)
    try:
        assert pt.selected_variant(512, 512, 2048) == pt.variant_by_name(simt[1])
        # (4096, 4096, 256) is at distance 1 from the second point and 8 from
        # the first: member 1's correction is (-0.3/64 + 0.3) / (1/64 + 1) > 0,
        # so member 0 wins there
        assert pt.selected_variant(4096, 4096, 256) == pt.variant_by_name(simt[0])
        del man["model"]["points"], man["model"]["resid"]
        json.dump(man, open(path, "w"))
        pt.load_manifest(path)
        assert pt.selected_variant(512, 512, 2048) == pt.variant_by_name(simt[0])  # a tie: the earlier member
    finally:
        pt.load_manifest(None)
