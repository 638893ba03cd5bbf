"""Pins of the plane split used to design the exact-plane GPU pins, and of
the input sets those pins use (CPU only).

The split (oracle/split.py) is checked against torch's FP32 -> BF16
conversion (round to nearest even, a library routine) and against values
worked by hand.  The input sets are then shown to exercise every product a
split-precision kernel keeps, to make every product it drops zero, and to
keep every partial sum an integer below 2^24, so that any summation order
in FP32 gives the exact result and a GPU result may be compared bit for bit.
"""

import numpy as np
import pytest

from oracle import gemm as og
from oracle.split import (BF16X3_DROPPED, BF16X3_KEPT, TF32X3_DROPPED, TF32X3_KEPT, bf16x3_planes,
                          f16_chunk_scales, f16x2_planes_scaled, round_sig, tf32x2_planes)
from workloads import matrix, rank1_operands, wide_int_operands

torch = pytest.importorskip("torch")


def _bits(x):
    return np.asarray(x, np.float32).view(np.uint32)


def test_round_sig_matches_torch_bfloat16():
    x = np.concatenate([matrix("uniform", 1, 1, 20000)[0], matrix("logu", 2, 1, 20000)[0],
                        np.float32([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 65793.0, 4095.0])])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(round_sig(x, 8), want)


def test_round_sig_hand_values():
    # ties go to the even significand
    assert round_sig(1 + 2 ** -8, 8) == 1.0
    assert round_sig(1 + 3 * 2 ** -8, 8) == 1 + 2 ** -6
    assert round_sig(1 + 2 ** -11, 11) == 1.0
    assert round_sig(1 + 3 * 2 ** -11, 11) == 1 + 2 ** -9
    assert round_sig(65793.0, 8) == 66048.0       # 65536 + 257: above the half-way point 256
    assert round_sig(4095.0, 11) == 4096.0
    assert round_sig(-3.0, 1) == -4.0 and round_sig(0.0, 8) == 0.0


@pytest.mark.parametrize("kind", ["uniform", "logu", "normal"])
def test_planes_sum_back_and_are_representable(kind):
    x = matrix(kind, 5, 1, 50000)[0]
    b = bf16x3_planes(x)
    assert np.array_equal(b[0] + b[1] + b[2], x.astype(np.float64))   # 24 bits = 8 + 8 + 8
    for p in b:
        assert np.all((_bits(p) & 0xFFFF) == 0)                        # BF16: low 16 bits zero
        assert np.array_equal(p.astype(np.float32).astype(np.float64), p)
    hi, lo = tf32x2_planes(x)
    assert np.all((_bits(hi) & 0x1FFF) == 0) and np.all((_bits(lo) & 0x1FFF) == 0)
    err = np.abs(x.astype(np.float64) - hi - lo)                      # 22 of 24 bits kept
    assert np.all(err <= np.abs(x) * 2.0 ** -21)


def _plane_products(A, B, pa, pb):
    """|A_i| @ |B_j| for every plane pair (i, j): entry (i, j) of the result
    is non-zero exactly when some term a_ik b_kj has non-zero planes i, j."""
    return {(i, j): np.abs(pa[i]) @ np.abs(pb[j]) for i in range(len(pa)) for j in range(len(pb))}


@pytest.mark.parametrize("M,N,K", [(300, 200, 128), (300, 200, 1024), (300, 136, 4096), (131, 97, 75)])
def test_wide_int_operands_exercise_every_kept_product(M, N, K):
    A, B, P = wide_int_operands(7, M, N, K)
    Ad, Bd = A.astype(np.float64), B.astype(np.float64)
    assert np.all(A == np.round(A)) and np.all(B == np.round(B))
    # every partial sum, in any order, is an integer of magnitude < 2^24
    assert (np.abs(Ad) @ np.abs(Bd)).max() < 2 ** 24
    exact = og.gemm(A, B)
    assert np.array_equal(exact, (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64))
    for planes, kept, dropped in ((bf16x3_planes, BF16X3_KEPT, BF16X3_DROPPED),
                                  (tf32x2_planes, TF32X3_KEPT, TF32X3_DROPPED)):
        pa, pb = planes(A), planes(B)
        prods = _plane_products(A, B, pa, pb)
        for ij in dropped:
            assert not prods[ij].any(), (planes.__name__, ij)     # nothing is lost
        for ij in kept:
            # each kept product is non-zero for a quarter of the outputs or more, so
            # a kernel that drops it gets many outputs wrong
            assert (prods[ij] > 0).mean() > 0.25, (planes.__name__, ij, (prods[ij] > 0).mean())
        # the kept products of the planes sum to the exact result
        total = sum(pa[i] @ pb[j] for (i, j) in kept)
        assert np.array_equal(total, exact)
        # plane partial sums stay below 2^24 too (the tensor core adds planes)
        pa_abs = sum(np.abs(p) for p in pa)
        pb_abs = sum(np.abs(p) for p in pb)
        assert (pa_abs @ pb_abs).max() < 2 ** 24
    if M >= P:
        # every k of A is non-zero in some row: all stages and chunks are exercised
        assert np.all((A != 0).any(axis=0))


@pytest.mark.parametrize("K", [128, 1024, 4096])
def test_rank1_operands_closed_form_and_planes(K):
    A, B = rank1_operands(5, 3, K)
    assert np.all(og.gemm(A, B) == K * (K - 1) / 2)
    assert K * (K - 1) / 2 < 2 ** 24
    b0, b1, b2 = bf16x3_planes(B)
    assert b1.any() == (K > 256) and not b2.any()   # k > 256 needs two BF16 planes, never three
    hi, lo = tf32x2_planes(B)
    assert lo.any() == (K > 2048)           # k >= 2048 needs more than 11 bits


def test_f16_chunk_scales_hand_values():
    X = np.zeros((5, 600))
    X[0, 5] = 1.0            # max 1: 2^14 * 1 in [2^14, 2^15)
    X[1, 0] = 3.0            # floor(log2 3) = 1 -> S = 13, 3 * 2^13 = 24576
    X[1, 599] = -2.0         # another chunk: S = 13 there as well
    X[2, 300] = -2.0 ** -60  # below the clamp: S = 63
    X[3, 599] = 2.0 ** 90    # above: S = -63
    S = f16_chunk_scales(X)  # chunks of 256 values of k
    assert S.shape == (5, 3)
    assert S[0, 0] == 14 and S[1, 0] == 13 and S[1, 2] == 13 and S[2, 1] == 63 and S[3, 2] == -63
    assert S[0, 1] == 63 and S[4, 0] == 63     # all-zero chunks
    G = f16_chunk_scales(X, group=32)          # one group of all five rows
    assert G.shape == (1, 3) and G[0, 0] == 13 and G[0, 2] == -63
    h0, h1, _ = f16x2_planes_scaled(X)
    assert h0[1, 0] == 24576.0 and h1[1, 0] == 0.0 and h0[1, 599] == -16384.0
    assert np.isinf(h0[3, 599])   # 2^90 * 2^-63 = 2^27 overflows FP16: outside the range


@pytest.mark.parametrize("kind", ["uniform", "logu", "normal"])
@pytest.mark.parametrize("group", [1, 32])
def test_f16_scaled_planes_error_bound(kind, group):
    X = matrix(kind, 9, 64, 1000)
    h0, h1, E = f16x2_planes_scaled(X, group)
    back = np.ldexp(h0 + h1, -E)
    # two 11-bit planes: error below 2^-21 of the value, plus half the FP16
    # subnormal spacing (2^-25 of the scaled unit) for values far below the
    # maximum of their group's chunk
    err = np.abs(X.astype(np.float64) - back)
    assert np.all(err <= np.abs(X) * 2.0 ** -21 + np.ldexp(2.0 ** -25, -E))
    assert np.all(np.abs(h0) <= 2 ** 15)   # rounding may reach 2^15; FP16 holds up to 65504


@pytest.mark.parametrize("M,N,K", [(300, 200, 1024), (300, 136, 4096)])
def test_wide_int_operands_under_the_scaled_f16_split(M, N, K):
    # The same input sets are exact for 3xF16: A's rows and B's column groups
    # split into two planes with nothing lost, the product h1 h1 is always
    # zero, and the three kept products are each non-zero for many outputs.
    A, B, _ = wide_int_operands(7, M, N, K)
    a0, a1, Ea = f16x2_planes_scaled(A)
    b0, b1, Eb = f16x2_planes_scaled(B.T, group=32)
    assert np.array_equal(np.ldexp(a0 + a1, -Ea), A.astype(np.float64))
    assert np.array_equal(np.ldexp(b0 + b1, -Eb), B.T.astype(np.float64))
    assert not (np.abs(a1) @ np.abs(b1).T).any()
    for pa, pb in ((a0, b0), (a0, b1), (a1, b0)):
        assert (np.abs(pa) @ np.abs(pb).T > 0).mean() > 0.25
