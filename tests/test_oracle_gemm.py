"""Pins of the CPU GEMM oracle against facts fixed by mathematics.

None of these compares the oracle with a retyped copy of itself: each case
has a result known independently (identity, permutation, exact integer
arithmetic, a closed-form sum, exact rationals, a library FP64 matmul) or an
invariant that a wrong index, dropped term, sign or transposed operand breaks.
"""

import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import normalised_error
from workloads import matrix


def _store(X, trans):
    """Storage for a logical matrix X under a transpose flag (row-major)."""
    return np.ascontiguousarray(X.T if trans == "T" else X)


TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


@pytest.mark.parametrize("ta,tb", TRANS)
def test_identity_gives_alpha_times_b(ta, tb):
    K, N = 37, 23
    B = matrix("uniform", 11, K, N)
    eye = np.eye(K, dtype=np.float32)
    out = og.gemm(_store(eye, ta), _store(B, tb), ta, tb, alpha=0.5)
    assert np.array_equal(out, 0.5 * B.astype(np.float64))


@pytest.mark.parametrize("ta,tb", TRANS)
def test_permutation_moves_rows_and_columns(ta, tb):
    M = 19
    rng = np.random.default_rng(3)
    p = rng.permutation(M)
    P = np.zeros((M, M), np.float32)
    P[np.arange(M), p] = 1.0          # (P X)[i] = X[p[i]]
    X = matrix("uniform", 12, M, 13)
    out = og.gemm(_store(P, ta), _store(X, tb), ta, tb)
    assert np.array_equal(out, X[p].astype(np.float64))
    Y = matrix("uniform", 13, 7, M)
    out2 = og.gemm(_store(Y, ta), _store(P, tb), ta, tb)  # (Y P)[:, j] = Y[:, q] with P[q, j] = 1
    q = np.argsort(p)
    assert np.array_equal(out2, Y[:, q].astype(np.float64))


@pytest.mark.parametrize("ta,tb", TRANS)
def test_small_integers_exact(ta, tb):
    M, N, K = 33, 29, 64
    A = matrix("ints", 21, M, K)
    B = matrix("ints", 22, K, N)
    Cin = matrix("ints", 23, M, N)
    exact = 3 * (A.astype(np.int64) @ B.astype(np.int64)) - 2 * Cin.astype(np.int64)
    out = og.gemm(_store(A, ta), _store(B, tb), ta, tb, alpha=3.0, beta=-2.0, C=Cin)
    assert np.array_equal(out, exact.astype(np.float64))


def test_rank_one_closed_form():
    # a_ik = 1, b_kj = k  =>  C_ij = sum_{k<K} k = K(K-1)/2, for every i, j.
    for K in (1, 2, 5, 64, 4096):
        A = np.ones((3, K), np.float32)
        B = np.repeat(np.arange(K, dtype=np.float32)[:, None], 4, axis=1)
        out = og.gemm(A, B)
        assert np.all(out == K * (K - 1) / 2), K


def test_sign_and_scale_closed_form():
    # a_ik = (-1)^k, b_kj = 1 => sum is 1 for odd K, 0 for even K.
    for K in (1, 2, 7, 10):
        A = np.array([[(-1.0) ** k for k in range(K)]], np.float32)
        B = np.ones((K, 2), np.float32)
        assert np.all(og.gemm(A, B, alpha=-4.0) == -4.0 * (K % 2))


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (5, 6, 3), (6, 1, 6), (4, 4, 6)])
@pytest.mark.parametrize("ta,tb", TRANS)
def test_tiny_exact_rationals(shape, ta, tb):
    M, N, K = shape
    A = matrix("logu", 31 + M, M, K)
    B = matrix("logu", 41 + N, K, N)
    Cin = matrix("uniform", 51, M, N)
    alpha, beta = np.float32(0.75), np.float32(-1.25)
    out = og.gemm(_store(A, ta), _store(B, tb), ta, tb, alpha=alpha, beta=beta, C=Cin)
    for i in range(M):
        for j in range(N):
            terms = [Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K)]
            exact = Fraction(float(alpha)) * sum(terms, Fraction(0)) + Fraction(float(beta)) * Fraction(float(Cin[i, j]))
            mag = float(abs(Fraction(float(alpha))) * sum(abs(t) for t in terms)) + abs(float(beta) * float(Cin[i, j]))
            # FP64 accumulation of K exact products plus the alpha/beta steps:
            # error <= (K + 2) * 2^-53 * magnitude (first-order bound).
            assert abs(out[i, j] - float(exact)) <= (K + 3) * 2.0 ** -53 * mag + 1e-300


@pytest.mark.parametrize("ta,tb", TRANS)
def test_agrees_with_library_fp64_matmul(ta, tb):
    M, N, K = 70, 45, 300
    A = matrix("uniform", 61, M, K)
    B = matrix("uniform", 62, K, N)
    ref = A.astype(np.float64) @ B.astype(np.float64)
    out = og.gemm(_store(A, ta), _store(B, tb), ta, tb)
    # Both are FP64 sums of exact products; they differ only by summation order.
    assert np.max(np.abs(out - ref)) <= K * 2.0 ** -52 * np.max(np.abs(A)) * np.max(np.abs(B)) * K


def test_beta_zero_ignores_nan_c():
    A = matrix("uniform", 71, 8, 9)
    B = matrix("uniform", 72, 9, 10)
    C = np.full((8, 10), np.nan, np.float32)
    out = og.gemm(A, B, beta=0.0, C=C)
    assert np.all(np.isfinite(out))


def test_rows_subset_matches_full():
    A = matrix("uniform", 81, 40, 17)
    B = matrix("uniform", 82, 17, 12)
    full = og.gemm(A, B)
    rows = [39, 0, 7, 7, 21]
    assert np.array_equal(og.gemm(A, B, rows=rows), full[rows])


def test_padded_leading_dimension():
    # Logical 9x5 inside 9x8 storage whose padding is NaN: padding is never read.
    A = matrix("uniform", 91, 9, 5, ld=8)
    B = matrix("uniform", 92, 5, 6)
    out = og.gemm(A, B, K=5)
    assert np.all(np.isfinite(out))
    assert np.array_equal(out, og.gemm(np.ascontiguousarray(A[:, :5]), B))


def test_empty_extents():
    A = np.zeros((0, 4), np.float32)
    B = np.zeros((4, 3), np.float32)
    assert og.gemm(A, B).shape == (0, 3)
    A = np.zeros((2, 0), np.float32)
    B = np.zeros((0, 3), np.float32)
    out = og.gemm(A, B, beta=0.0)
    assert np.array_equal(out, np.zeros((2, 3)))


def test_normalised_error_definition():
    C_ref = np.array([[1.0, -2.0]])
    C = np.array([[1.0, -2.5]])
    # denom = K*maxA*maxB*|alpha| + |beta|*maxC = 4*1*2*1 + 0 = 8
    assert normalised_error(C, C_ref, 4, 1.0, 2.0) == pytest.approx(0.5 / 8)
    assert normalised_error(C, C_ref, 4, 1.0, 2.0, alpha=2.0, beta=1.0, maxC=4.0) == pytest.approx(0.5 / 20)
    assert normalised_error(np.array([[np.nan]]), np.array([[0.0]]), 1, 1, 1) == float("inf")


# --- planted mistakes: each mutation of the C source must fail some pin ------

MUTATIONS = [
    ("k * lda + i", "i * lda + k"),                    # transposed-A index
    ("j * ldb + k", "k * ldb + j"),                    # transposed-B index
    ("for (long k = 0; k < K; ++k)", "for (long k = 1; k < K; ++k)"),  # dropped term
    ("v += beta *", "v -= beta *"),                    # wrong sign
    ("acc[j] += a *", "acc[j] = a *"),                 # no accumulation
]


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_planted_mistakes_are_caught(old, new, monkeypatch):
    src = open(og._build.SRC).read()
    assert old in src
    tmp = tempfile.mkdtemp()
    try:
        path = os.path.join(tmp, "gemm_ref.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new, 1))
        lib = os.path.join(tmp, "_gemm_ref.so")
        subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", path, "-o", lib],
                       check=True, capture_output=True)
        monkeypatch.setattr(og, "_lib", None)
        monkeypatch.setattr(og._build, "build", lambda force=False: lib)
        pins = [
            lambda: test_small_integers_exact("N", "T"),
            lambda: test_small_integers_exact("T", "N"),
            lambda: test_rank_one_closed_form(),
            lambda: test_identity_gives_alpha_times_b("T", "T"),
        ]
        failures = 0
        for pin in pins:
            try:
                pin()
            except AssertionError:
                failures += 1
        assert failures > 0, "mutation %r -> %r survived every pin" % (old, new)
    finally:
        og._lib = None
        shutil.rmtree(tmp, ignore_errors=True)
