"""Pins of the portability-tuning oracle (selection arithmetic)."""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import select as osel

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_hand_worked_tiny_table():
    g = _load("select_tiny.json")
    t = np.array(g["times"])
    assert list(osel.per_shape_best(t)) == g["t_best"]
    for k, opt in g["optimum"].items():
        kappa, val = osel.portability_tune_exhaustive(t, int(k), range(t.shape[1]))
        assert kappa == opt["kappa"], k
        assert val == pytest.approx(opt["value"], rel=1e-12)


def test_table5_post_processing_arithmetic():
    g = _load("table5_quadro.json")
    slow, best = g["rows"]
    t_best = best["runtime_ms"]
    assert round(osel.slowdown_vs_best(best["runtime_ms"], t_best), 2) == best["slowdown_vs_oracle"]
    assert round(osel.slowdown_vs_best(slow["runtime_ms"], t_best), 2) == slow["slowdown_vs_oracle"]
    # Worst time implied by the best row, then the slow row's speedup from it.
    t_worst = t_best * best["speedup_vs_worst"]
    assert round(osel.speedup_vs_worst(slow["runtime_ms"], t_worst), 2) == slow["speedup_vs_worst"]
    # The two rows imply the same worst time to within print rounding.
    assert abs(slow["runtime_ms"] * slow["speedup_vs_worst"] - t_worst) / t_worst < 1e-3


def test_post_processing_on_a_table():
    t = np.array([[2.0, 9.0], [4.0, 3.0], [np.inf, 6.0]])
    assert list(osel.per_shape_best(t)) == [2.0, 3.0]
    assert list(osel.per_shape_worst(t)) == [4.0, 9.0]
    assert osel.autotune(t, 0) == 0 and osel.autotune(t, 1) == 1


def test_search_space_count_section_iv_c():
    # 1,343 Quadro variants, best 3, 10 inputs: "over 24 billion" evaluations.
    n = osel.search_space_evaluations(10, 1343, 3)
    assert n == 10 * 1343 ** 3
    assert 24e9 < n < 25e9


def _random_table(seed, V, S, invalid=0.1):
    rng = np.random.default_rng(seed)
    t = np.exp(rng.normal(0, 0.6, size=(V, S)))
    t[rng.random((V, S)) < invalid] = np.inf
    for s in range(S):  # every shape keeps at least one valid variant
        if not np.isfinite(t[:, s]).any():
            t[0, s] = 1.0
    return t


@pytest.mark.parametrize("seed", range(6))
def test_invariants(seed):
    t = _random_table(seed, 7, 9)
    shapes = range(9)
    cand = osel.candidate_variants(t, shapes)
    vals = [osel.portability_tune_exhaustive(t, k, shapes)[1] for k in range(1, len(cand) + 1)]
    assert all(b >= a - 1e-15 for a, b in zip(vals, vals[1:])), "monotone in k"
    assert vals[-1] == pytest.approx(1.0, rel=1e-12), "all variants reach every t_best"
    assert all(0.0 <= v <= 1.0 + 1e-12 for v in vals)
    # k = 1 is the single variant with the best geomean performance.
    perf = osel.per_shape_best(t)[None, :] / t
    single = []
    for v in range(t.shape[0]):
        p = perf[v]
        single.append(0.0 if np.any(p == 0) else float(np.exp(np.mean(np.log(p)))))
    assert vals[0] == pytest.approx(max(single), rel=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_exhaustive_equals_brute_force_over_ordered_tuples(seed):
    # Independent enumeration: ordered k-tuples with repetition (the paper's
    # |K|^|kappa| space), scored with a vectorised min.
    t = _random_table(100 + seed, 6, 8, invalid=0.0)
    tb = t.min(axis=0)
    for k in (1, 2, 3):
        best = -1.0
        for tup in itertools.product(range(6), repeat=k):
            m = t[list(tup)].min(axis=0)
            best = max(best, float(np.exp(np.mean(np.log(tb / m)))))
        _, val = osel.portability_tune_exhaustive(t, k, range(8))
        assert val == pytest.approx(best, rel=1e-12)


def test_planted_block_structure():
    # Variant g is fastest (1.0) on shape group g and slow (8.0) elsewhere;
    # variant 4 is 2.0 everywhere.  With k = 4 the specialists are optimal
    # (value 1); with k = 1 the generalist wins (value 1/2 vs 8^(-3/4)).
    groups = [[0, 1], [2, 3], [4, 5], [6, 7]]
    t = np.full((5, 8), 8.0)
    for g, ss in enumerate(groups):
        t[g, ss] = 1.0
    t[4, :] = 2.0
    kappa, val = osel.portability_tune_exhaustive(t, 4, range(8))
    assert kappa == [0, 1, 2, 3] and val == pytest.approx(1.0)
    kappa, val = osel.portability_tune_exhaustive(t, 1, range(8))
    assert kappa == [4] and val == pytest.approx(0.5)
    # Scored on a subset of shapes only.
    assert osel.set_performance(t, [0], [0, 1]) == pytest.approx(1.0)
    assert osel.set_performance(t, [0], [2, 3]) == pytest.approx(1.0 / 8)


def test_invalid_everywhere_in_set_scores_zero():
    t = np.array([[1.0, np.inf], [2.0, 2.0]])
    assert osel.set_performance(t, [0], [0, 1]) == 0.0
    assert osel.set_performance(t, [0, 1], [0, 1]) == pytest.approx(1.0)


def test_nearest_shape_rule():
    shapes = [(128, 128, 128), (1024, 1024, 1024), (4096, 128, 512)]
    assert osel.nearest_shape((1024, 1024, 1024), shapes) == 1
    assert osel.nearest_shape((2048, 1024, 1024), shapes) == 1      # distance 1 vs 7+ vs ...
    assert osel.nearest_shape((4096, 256, 512), shapes) == 2
    # Equidistant (log2 distance 3.5 to both (128^3) and (1024^3)): lower index wins.
    m = int(round(2 ** 8.5))
    d0 = sum(abs(math.log2(x) - 7) for x in (m, 128, 1024))
    d1 = sum(abs(math.log2(x) - 10) for x in (m, 128, 1024))
    q = (m, 128, 1024)
    assert osel.nearest_shape(q, shapes[:2]) == (0 if d0 <= d1 else 1)


def test_best_in_set_ties_go_to_lowest_id():
    t = np.array([[3.0], [1.0], [1.0]])
    assert osel.best_in_set(t, [2, 1, 0], 0) == 1


# ---- alternative selections (Section IV-C): k-means and regression tree ---------------

def _feat(shapes):
    return [tuple(math.log2(x) for x in sh) for sh in shapes]


@pytest.mark.parametrize("seed", range(4))
def test_kmeans_single_cluster_is_best_mean_performance(seed):
    t = _random_table(200 + seed, 7, 9, invalid=0.1)
    ids, assign = osel.kmeans_select(t, 1, range(9), seed=seed)
    perf = np.where(np.isfinite(t), osel.per_shape_best(t)[None, :] / t, 0.0)
    assert ids == [int(np.argmax(perf.mean(axis=1)))]
    assert set(assign) == {0}


def test_kmeans_one_cluster_per_shape_recovers_per_shape_best():
    # Every shape has a different best variant (all points distinct).
    t = np.full((5, 5), 4.0)
    for s in range(5):
        t[s, s] = 1.0
    t[0, 1] = 2.0
    ids, _ = osel.kmeans_select(t, 5, range(5), seed=3)
    assert ids == sorted({osel.autotune(t, s) for s in range(5)}) == [0, 1, 2, 3, 4]


def test_kmeans_planted_clusters():
    # Shapes 0-3 favour variant 2, shapes 4-7 favour variant 5, strongly.
    rng = np.random.default_rng(0)
    t = 3.0 + rng.random((6, 8))
    t[2, :4] = 1.0
    t[5, 4:] = 1.0
    for seed in range(5):
        ids, assign = osel.kmeans_select(t, 2, range(8), seed=seed)
        assert ids == [2, 5]
        assert len(set(assign[:4])) == 1 and len(set(assign[4:])) == 1 and assign[0] != assign[4]


def test_tree_single_leaf_is_best_mean_performance():
    t = _random_table(300, 6, 8)
    shapes = [(2 ** (7 + s % 4), 2 ** (7 + s // 4), 256) for s in range(8)]
    ids, leaves = osel.tree_select(t, 1, range(8), _feat(shapes))
    perf = np.where(np.isfinite(t), osel.per_shape_best(t)[None, :] / t, 0.0)
    assert ids == [int(np.argmax(perf.mean(axis=1)))]
    assert len(leaves) == 1


def test_tree_planted_split_on_m():
    # M <= 512 -> variant 0 is best, M > 512 -> variant 1; N, K are noise.
    shapes = [(m, n, k) for m in (128, 512, 1024, 4096) for n in (128, 4096) for k in (256, 2048)]
    t = np.full((3, len(shapes)), 2.0)
    for s, (m, n, k) in enumerate(shapes):
        t[0 if m <= 512 else 1, s] = 1.0
        t[2, s] = 1.5 + 0.01 * (n == 4096)
    ids, leaves = osel.tree_select(t, 2, range(len(shapes)), _feat(shapes))
    assert ids == [0, 1]
    assert sorted(len(ix) for ix, _ in leaves) == [8, 8]
    for ix, v in leaves:
        assert {shapes[i][0] <= 512 for i in ix} == {v == 0}


def test_tree_first_split_maximises_error_reduction_by_brute_force():
    t = _random_table(400, 5, 10, invalid=0.0)
    feats = [(float(a), float(b)) for a, b in np.random.default_rng(4).integers(0, 5, size=(10, 2))]
    _, leaves = osel.tree_select(t, 2, range(10), feats)
    perf = osel.per_shape_best(t)[None, :] / t  # (V, S)
    pts = perf.T

    def sse(ix):
        return float(((pts[ix] - pts[ix].mean(axis=0)) ** 2).sum()) if len(ix) else 0.0

    best = None
    for f in range(2):
        for thr in sorted({x[f] for x in feats}):
            left = [i for i in range(10) if feats[i][f] <= thr]
            right = [i for i in range(10) if feats[i][f] > thr]
            if left and right:
                gain = sse(list(range(10))) - sse(left) - sse(right)
                best = gain if best is None else max(best, gain)
    got = sse(list(range(10))) - sse(leaves[0][0]) - sse(leaves[1][0])
    assert got == pytest.approx(best, rel=1e-9)


# ---- time model of the runtime selector (the reading for shapes outside the table) ----

def _grid(levels=(128, 512, 1024, 4096)):
    return [(m, n, k) for m in levels for n in levels for k in levels]


def test_model_recovers_a_planted_quadratic():
    rng = np.random.default_rng(11)
    shapes = _grid()
    beta = rng.normal(0, 1, osel.MODEL_FEATURES)
    times = [math.exp(float(np.dot(beta, osel.model_features(s)))) for s in shapes]
    c = osel.model_fit(times, shapes)
    assert np.allclose(c, beta, rtol=0, atol=1e-9)


def test_model_degrades_to_linear_then_mean():
    rng = np.random.default_rng(12)
    shapes = [(128, 512, 1024), (4096, 512, 128), (512, 4096, 512), (1024, 128, 4096), (256, 256, 256)]
    beta = np.concatenate([rng.normal(0, 1, 4), np.zeros(6)])
    times = [math.exp(float(np.dot(beta, osel.model_features(s)))) for s in shapes]
    c = osel.model_fit(times, shapes)            # 5 points: the quadratic is not determined
    assert np.allclose(c, beta, atol=1e-9)
    c2 = osel.model_fit([2.0, 8.0, math.inf], shapes[:3])   # 2 valid points: the mean of ln t
    assert c2[0] == pytest.approx(math.log(4.0)) and not any(c2[1:])
    assert osel.model_fit([math.inf] * 3, shapes[:3]) is None
    # dependent columns (every shape has the same N): no linear model either, the mean
    same_n = [(m, 512, k) for m in (128, 512, 1024, 4096) for k in (128, 512, 1024)]
    c3 = osel.model_fit([float(i + 1) for i in range(len(same_n))], same_n)
    assert c3[0] == pytest.approx(float(np.mean(np.log(np.arange(1, 13))))) and not any(c3[1:])


def test_model_pick_is_the_argmin_of_the_models():
    rng = np.random.default_rng(13)
    coefs = [list(rng.normal(0, 1, osel.MODEL_FEATURES)) for _ in range(5)]
    coefs[2] = None
    for q in [(300, 700, 2000), (128, 4096, 128), (5000, 100, 900)]:
        f = np.array(osel.model_features(q))
        preds = [np.dot(c, f) if c is not None else np.inf for c in coefs]
        assert osel.model_pick(coefs, q) == int(np.argmin(preds))
    # ties go to the earlier member; no model at all gives None
    same = [1.0] + [0.0] * 9
    assert osel.model_pick([same, same], (512, 512, 512)) == 0
    assert osel.model_pick([None, None], (512, 512, 512)) is None


def test_model_features_closed_form():
    # log2 512 = 9 is the centre; 4096 and 64 sit one scale unit (3 octaves) away.
    assert osel.model_features((512, 512, 512)) == [1.0] + [0.0] * 9
    assert osel.model_features((4096, 64, 512)) == [1.0, 1.0, -1.0, 0.0, 1.0, 1.0, 0.0, -1.0, 0.0, 0.0]


def test_residual_correction_closed_forms():
    # Intercept-only model ln t = 1 and two training shapes with residuals
    # r1 = 0.5 at distance 1 and r2 = -1.0 at distance 2 from the query:
    # weights 1 and 1/4, so the correction is (0.5 - 0.25) / 1.25 = 0.2.
    coef = [1.0] + [0.0] * 9
    q = (512, 512, 512)
    points = [(1024, 512, 512), (512, 2048, 512)]   # log2 distances 1 and 2
    assert osel.log_distance(q, points[0]) == 1.0 and osel.log_distance(q, points[1]) == 2.0
    assert osel.model_predict(coef, q, [0.5, -1.0], points) == pytest.approx(1.2)
    # an invalid point (None) does not count; one valid point gives its residual
    assert osel.model_predict(coef, q, [None, -1.0], points) == pytest.approx(0.0)
    # at distance 0 the prediction is that shape's measured ln t
    times = [math.e ** 2, math.e ** 0.25]
    res = osel.model_residuals(coef, times, points)
    assert res == pytest.approx([1.0, -0.75])
    assert osel.model_predict(coef, points[1], res, points) == pytest.approx(0.25)
    # residuals of an exactly quadratic member are zero: no change to the pick
    rng = np.random.default_rng(14)
    shapes = _grid()
    coefs, resids = [], []
    for _ in range(4):
        beta = rng.normal(0, 1, osel.MODEL_FEATURES)
        t = [math.exp(float(np.dot(beta, osel.model_features(s)))) for s in shapes]
        c = osel.model_fit(t, shapes)
        coefs.append(c)
        resids.append(osel.model_residuals(c, t, shapes))
        assert np.allclose([r for r in resids[-1]], 0.0, atol=1e-9)
    for q in [(300, 700, 2000), (128, 4096, 200), (5000, 100, 900)]:
        assert osel.model_pick(coefs, q, resids, shapes) == osel.model_pick(coefs, q)


def test_residual_correction_can_change_the_pick():
    # Two members with the same model; member 1 is measured 0.3 faster than
    # its model at the training shape next to the query and 0.3 slower far
    # away, so the nearby residual wins and member 1 is picked.
    coef = [0.0] * 10
    points = [(512, 512, 1024), (4096, 4096, 128)]
    q = (512, 512, 2048)                      # distances 1 and 3 + 3 + 4 = 10
    resids = [[0.0, 0.0], [-0.3, 0.3]]
    assert osel.model_pick([coef, coef], q) == 0          # a tie without residuals
    assert osel.model_pick([coef, coef], q, resids, points) == 1
