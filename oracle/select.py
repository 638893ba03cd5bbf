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
