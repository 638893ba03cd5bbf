"""Portability-tuning arithmetic, written plainly (test infrastructure only).

A timing table is an array ``times[v, s]`` (variant v, shape s) in any time
unit, with ``inf`` for a variant that is invalid or failed on that shape.

Names follow the paper:

* AutoTune (Section IV-A): on one device the single best variant for one
  input, i.e. the per-shape argmin.  Its time is the "Oracle" of the
  evaluation (Section V-E), called ``t_best`` here to keep it apart from the
  CPU GEMM oracle.
* PortabilityTune (Section IV-B): a set kappa of at most k variants for a set
  of inputs.
* Library cost function (Section IV-D, Eq. 1).  As printed, the fraction has
  the max of the set's runtimes over the Oracle, which would reward slower
  kernels; the reading used here (the text around Eq. 1 and the S/O figure of
  merit) is the performance of kappa on shape s,
      perf(kappa, s) = t_best(s) / min_{v in kappa} t(v, s)   in (0, 1],
  summarised by the geometric mean over shapes and maximised.  Its reciprocal
  is the geomean Slowdown over Oracle (S/O).
* Post-processing (Section V-D, Table 5): slowdown vs the Oracle t/t_best and
  speedup vs the worst variant t_worst/t.
* Exhaustive search cost (Section IV-C): |inputs| * |K|^|kappa| evaluations
  (ordered tuples).
"""

from __future__ import annotations

import itertools
import math

import numpy as np


def per_shape_best(times: np.ndarray) -> np.ndarray:
    """t_best[s] = min over all variants of times[v, s] (the paper's Oracle)."""
    return np.min(np.asarray(times, dtype=np.float64), axis=0)


def per_shape_worst(times: np.ndarray) -> np.ndarray:
    """Slowest valid time per shape (inf entries ignored)."""
    t = np.asarray(times, dtype=np.float64)
    masked = np.where(np.isfinite(t), t, -np.inf)
    return np.max(masked, axis=0)


def autotune(times: np.ndarray, s: int) -> int:
    """AutoTune on one device: argmin_v times[v, s], ties -> lowest id."""
    col = np.asarray(times, dtype=np.float64)[:, s]
    best = None
    for v in range(col.shape[0]):
        if best is None or col[v] < col[best]:
            best = v
    return int(best)


def slowdown_vs_best(t: float, t_best: float) -> float:
    """Table 5 column 'Slowdown vs Oracle'."""
    return t / t_best


def speedup_vs_worst(t: float, t_worst: float) -> float:
    """Table 5 column 'Speedup vs Worst'."""
    return t_worst / t


def search_space_evaluations(n_inputs: int, n_variants: int, k: int) -> int:
    """Evaluations of an exhaustive search over ordered k-tuples (Section IV-C)."""
    return n_inputs * n_variants ** k


def perf_of_set(times: np.ndarray, kappa, s: int, t_best=None) -> float:
    """t_best(s) / min_{v in kappa} t(v, s); 0 when no member is valid on s."""
    t = np.asarray(times, dtype=np.float64)
    tb = per_shape_best(t) if t_best is None else t_best
    m = min(t[v, s] for v in kappa)
    if not math.isfinite(m):
        return 0.0
    return float(tb[s] / m)


def set_performance(times: np.ndarray, kappa, shapes) -> float:
    """Eq. 1 (reading above): geomean over ``shapes`` of perf(kappa, s).

    t_best is taken over every variant of the table, not only kappa.  The log
    terms are summed in the order of ``shapes``.
    """
    t = np.asarray(times, dtype=np.float64)
    tb = per_shape_best(t)
    shapes = list(shapes)
    if not shapes:
        return 1.0
    total = 0.0
    for s in shapes:
        p = perf_of_set(t, kappa, s, tb)
        if p <= 0.0:
            return 0.0
        total += math.log(p)
    return math.exp(total / len(shapes))


def candidate_variants(times: np.ndarray, shapes) -> list:
    """Variants valid (finite time) on at least one of ``shapes``."""
    t = np.asarray(times, dtype=np.float64)
    shapes = list(shapes)
    return [v for v in range(t.shape[0]) if any(math.isfinite(t[v, s]) for s in shapes)]


def portability_tune_exhaustive(times: np.ndarray, k: int, shapes):
    """PortabilityTune by enumerating every k-subset of the candidates.

    Returns (kappa as a sorted list of ids, its Eq. 1 value).  Subsets are
    visited in lexicographic order and a later subset replaces the current
    best only if strictly better, so among exact ties the lexicographically
    smallest set wins.  When k is at least the number of candidates, every
    candidate is returned.
    """
    shapes = list(shapes)
    cand = candidate_variants(times, shapes)
    if k >= len(cand):
        return cand, set_performance(times, cand, shapes)
    best_set, best_val = None, -1.0
    for combo in itertools.combinations(cand, k):
        val = set_performance(times, combo, shapes)
        if val > best_val:
            best_set, best_val = list(combo), val
    return best_set, best_val


def best_in_set(times: np.ndarray, kappa, s: int) -> int:
    """The member of kappa with the smallest time on shape s (ties -> lowest id)."""
    t = np.asarray(times, dtype=np.float64)
    best = None
    for v in sorted(kappa):
        if best is None or t[v, s] < t[best, s]:
            best = v
    return int(best)


def nearest_shape(query, shapes) -> int:
    """Runtime-selector rule for a shape outside the table.

    The nearest listed shape in (log2 M, log2 N, log2 K) under the L1
    distance; ties go to the lower index.  An exact match has distance 0.
    """
    q = [math.log2(x) for x in query]
    best, best_d = None, None
    for i, sh in enumerate(shapes):
        d = sum(abs(math.log2(a) - b) for a, b in zip(sh, q))
        if best_d is None or d < best_d:
            best, best_d = i, d
    return best


# ---- time model for shapes outside the table ------------------------------------------
#
# The paper leaves inference for unlisted inputs open (Section V-G).  The
# reading taken here: for every member of kappa, ln(time) is modelled as a
# quadratic in the centred log-extents u = (log2 M - 9) / 3, v = (log2 N -
# 9) / 3, w = (log2 K - 9) / 3, fitted by least squares on the training
# shapes where the member is valid; the selector takes the member with the
# smallest predicted time (ties to the earlier member).  With too few
# training points for the quadratic (fewer than 10, or dependent columns)
# the linear model in (1, u, v, w) is used, with fewer than that the mean.

MODEL_FEATURES = 10


def model_features(shape) -> list:
    """[1, u, v, w, u^2, v^2, w^2, uv, uw, vw] of shape (M, N, K)."""
    u, v, w = ((math.log2(x) - 9.0) / 3.0 for x in shape[:3])
    return [1.0, u, v, w, u * u, v * v, w * w, u * v, u * w, v * w]


def _full_rank(X) -> bool:
    # Same criterion as the library's QR: every |R_ii| above 1e-9 of the largest.
    r = np.abs(np.diag(np.linalg.qr(X, mode="r")))
    return bool(len(r) == X.shape[1] and np.all(r > 1e-9 * r.max()))


def model_fit(times_row, train_shapes):
    """Coefficients (length 10) of one variant's ln-time model over the
    training shapes, or None when the variant is valid on none of them."""
    pts = [(model_features(sh), math.log(t)) for sh, t in zip(train_shapes, times_row)
           if np.isfinite(t) and t > 0]
    if not pts:
        return None
    X = np.array([f for f, _ in pts])
    y = np.array([v for _, v in pts])
    for p in (MODEL_FEATURES, 4):
        if len(pts) >= p and _full_rank(X[:, :p]):
            c = np.linalg.lstsq(X[:, :p], y, rcond=None)[0]
            return [float(x) for x in c] + [0.0] * (MODEL_FEATURES - p)
    return [float(np.mean(y))] + [0.0] * (MODEL_FEATURES - 1)


def model_residuals(coef, times_row, train_shapes):
    """ln t - model at every training shape (None where the variant is
    invalid there); None when the variant has no model."""
    if coef is None:
        return None
    out = []
    for sh, t in zip(train_shapes, times_row):
        if np.isfinite(t) and t > 0:
            out.append(math.log(t) - float(np.dot(np.array(coef), np.array(model_features(sh)))))
        else:
            out.append(None)
    return out


def log_distance(a, b) -> float:
    """L1 distance of two shapes in (log2 M, log2 N, log2 K)."""
    return sum(abs(math.log2(x) - math.log2(y)) for x, y in zip(a[:3], b[:3]))


def model_predict(coef, query, resid=None, points=None) -> float:
    """Predicted ln-time of one member at `query`: the quadratic model plus,
    when residuals are given, their weighted mean over the training shapes
    where the member is valid, with weights 1 / d^2 (d = log_distance).  A
    query at distance 0 from valid training shapes takes the mean residual
    of those shapes, so the prediction there is their measured ln-time."""
    pred = float(np.dot(np.array(coef), np.array(model_features(query))))
    if resid is None:
        return pred
    pts = [(log_distance(query, q), r) for q, r in zip(points, resid) if r is not None]
    if not pts:
        return pred
    at = [r for d, r in pts if d == 0.0]
    if at:
        return pred + sum(at) / len(at)
    num = sum(r / (d * d) for d, r in pts)
    den = sum(1.0 / (d * d) for d, r in pts)
    return pred + num / den


def model_pick(coefs, query, resids=None, points=None):
    """Index of the member with the smallest predicted ln-time at `query`
    (ties to the earlier member); None when no member has a model.  With
    `resids` (one list per member, aligned with `points`) the predictions
    carry the residual correction of model_predict."""
    best, bp = None, None
    for i, c in enumerate(coefs):
        if c is None:
            continue
        pred = model_predict(c, query, None if resids is None else resids[i], points)
        if bp is None or pred < bp:
            best, bp = i, pred
    return best


# ---- alternative selections (Section IV-C) ---------------------------------------------
#
# Both work on the training shapes' performance vectors: shape s is the point
# perf[:, s] with perf[v, s] = t_best(s) / t(v, s) (0 where v is invalid), a
# point in |K|-dimensional space (one coordinate per variant).
#
# Random draws come from SplitMix64 (the same published definition as the
# input generator): draw i of seed `seed` is mix(seed + (i + 1) * gamma);
# u = (x >> 11) * 2^-53 is uniform on [0, 1).

def _splitmix_u(seed: int, i: int) -> float:
    m = (1 << 64) - 1
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    z = z ^ (z >> 31)
    return (z >> 11) * 2.0 ** -53


def performance_vectors(times: np.ndarray, shapes) -> list:
    """points[j][v] = t_best(s_j) / t(v, s_j), 0 for an invalid entry (plain lists)."""
    t = np.asarray(times, dtype=np.float64)
    tb = per_shape_best(t)
    pts = []
    for s in shapes:
        pts.append([float(tb[s] / t[v, s]) if math.isfinite(t[v, s]) else 0.0 for v in range(t.shape[0])])
    return pts


def _sqdist(a, b) -> float:
    d = 0.0
    for x, y in zip(a, b):
        d += (x - y) * (x - y)
    return d


def _argmax_first(vec) -> int:
    best = 0
    for v in range(1, len(vec)):
        if vec[v] > vec[best]:
            best = v
    return best


def kmeans_select(times: np.ndarray, k: int, shapes, seed: int = 0, max_iter: int = 100):
    """k-means selection (Section IV-C-2).

    Points: the training shapes' performance vectors.  Initial centroids by
    k-means++ (first point: floor(u_0 * n); each next point with probability
    proportional to its squared distance to the nearest chosen centroid,
    using draw 1, 2, ...; if every distance is 0, the lowest unchosen index).
    Lloyd iterations: each point to its nearest centroid (ties to the lower
    centroid), centroids = cluster means (an empty cluster keeps its
    centroid), until no assignment changes or max_iter.  Each centroid then
    contributes its highest-performing variant (ties to the lower id).
    Returns (sorted distinct variant ids, final assignment of the points).
    """
    pts = performance_vectors(times, shapes)
    n = len(pts)
    k = min(k, n)
    draws = 0
    first = int(_splitmix_u(seed, draws) * n) if n else 0
    draws += 1
    centers = [list(pts[first])]
    chosen = [first]
    while len(centers) < k:
        d2 = [min(_sqdist(p, c) for c in centers) for p in pts]
        total = 0.0
        for x in d2:
            total += x
        if total <= 0.0:
            nxt = next(i for i in range(n) if i not in chosen)
        else:
            u = _splitmix_u(seed, draws) * total
            acc, nxt = 0.0, n - 1
            for i, x in enumerate(d2):
                acc += x
                if acc > u:
                    nxt = i
                    break
        draws += 1
        chosen.append(nxt)
        centers.append(list(pts[nxt]))
    assign = [-1] * n
    for _ in range(max_iter):
        changed = False
        for i, p in enumerate(pts):
            best, bd = 0, _sqdist(p, centers[0])
            for c in range(1, len(centers)):
                d = _sqdist(p, centers[c])
                if d < bd:
                    best, bd = c, d
            if assign[i] != best:
                assign[i] = best
                changed = True
        if not changed:
            break
        for c in range(len(centers)):
            members = [pts[i] for i in range(n) if assign[i] == c]
            if members:
                dim = len(members[0])
                mean = [0.0] * dim
                for m in members:
                    for v in range(dim):
                        mean[v] += m[v]
                centers[c] = [x / len(members) for x in mean]
    ids = sorted({_argmax_first(c) for c in centers})
    return ids, assign


def tree_select(times: np.ndarray, k: int, shapes, features):
    """Regression-tree selection (Section IV-C-3).

    A regression tree maps an environment's features (here the log2 of its
    M, N, K) to its performance vector, with squared error summed over the
    vector's coordinates.  It is grown best-first: the leaf whose best split
    removes the most squared error is split next, until it has k leaves or no
    split removes any error.  Candidate splits: every feature, thresholds
    halfway between consecutive distinct values; ties go to the lower feature
    index, then the lower threshold, then the earlier leaf.  Each leaf
    contributes the highest-performing variant of its mean vector (ties to
    the lower id).  Returns (sorted distinct ids, leaves) with leaves a list
    of (member point indices, variant).
    """
    pts = performance_vectors(times, shapes)
    feats = [list(features[s]) for s in shapes]
    dim = len(pts[0]) if pts else 0

    def sse(idx):
        if not idx:
            return 0.0
        mean = [0.0] * dim
        for i in idx:
            for v in range(dim):
                mean[v] += pts[i][v]
        mean = [x / len(idx) for x in mean]
        e = 0.0
        for i in idx:
            e += _sqdist(pts[i], mean)
        return e

    def best_split(idx):
        base = sse(idx)
        best = None  # (gain, feature, threshold, left, right)
        for f in range(len(feats[0]) if feats else 0):
            vals = sorted({feats[i][f] for i in idx})
            for a, b in zip(vals, vals[1:]):
                thr = 0.5 * (a + b)
                left = [i for i in idx if feats[i][f] <= thr]
                right = [i for i in idx if feats[i][f] > thr]
                gain = base - sse(left) - sse(right)
                if best is None or gain > best[0]:
                    best = (gain, f, thr, left, right)
        return best

    leaves = [list(range(len(pts)))]
    while len(leaves) < k:
        cand = None
        for li, idx in enumerate(leaves):
            b = best_split(idx)
            if b is not None and b[0] > 0.0 and (cand is None or b[0] > cand[0][0]):
                cand = (b, li)
        if cand is None:
            break
        (gain, f, thr, left, right), li = cand
        leaves[li:li + 1] = [left, right]
    out = []
    for idx in leaves:
        mean = [0.0] * dim
        for i in idx:
            for v in range(dim):
                mean[v] += pts[i][v]
        out.append((idx, _argmax_first(mean)))
    return sorted({v for _, v in out}), out
