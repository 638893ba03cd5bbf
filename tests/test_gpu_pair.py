"""GPU: the two-CTA (cta_group::2) tensor-core versions.

A cluster of two CTAs computes a 256 x 128 or 256 x 256 tile: each CTA loads
its 128 rows of A and half of the tile's columns of B, the even CTA issues
M = 256 MMAs over both CTAs' shared memory, and each CTA drains its own rows
from its own tensor memory.  These tests hold the pair versions to the FP64
oracle where the pairing can go wrong: row tiles whose second half lies
partly or wholly past M (the odd CTA then loads zero rows and stores
nothing), N not a multiple of the per-CTA half, more tiles than resident
pairs, every transpose pair, alpha/beta, and the all-plane exact pins of the
split.  The 256-column pairs also run stream-K over CTA pairs (each CTA of a
finishing pair adds the partial tiles of the same-rank CTAs of earlier
pairs): the `_stk` version always, the hybrid when the last wave of pair
tiles is under 3/4 full.
"""

import numpy as np
import pytest

from oracle import gemm as og
from workloads import matrix, wide_int_operands

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
PAIRS = ("tc3xf16_m256n128_p4_2sm", "tc3xtf32_m256n128_p4_2sm", "tc3xf16_m256n256_p6_sw64_2sm",
         "tc3xf16_m256n256_p5_sw64_2sm", "tc3xf16_m256n256_p6_sw64_2sm_stk")


def _vid(name):
    return pt.variant_by_name(name)


def _run(name, A, B, M, N, ta="N", tb="N", alpha=1.0, beta=0.0, C0=None):
    Ad, Bd = torch.from_numpy(np.ascontiguousarray(A)).to(DEV), torch.from_numpy(np.ascontiguousarray(B)).to(DEV)
    C = torch.from_numpy(C0.copy()).to(DEV) if C0 is not None else torch.full((M, N), float("nan"), device=DEV)
    pt.sgemm(Ad, Bd, C, alpha=alpha, beta=beta, transA=ta, transB=tb, variant=_vid(name))
    torch.cuda.synchronize()
    return C.cpu().numpy()


def test_pair_versions_registered():
    for name in PAIRS:
        d = pt.variant(_vid(name))
        bn = 256 if "n256" in name else 128
        assert d["bm"] == 256 and d["bn"] == bn and d["trans_mask"] == 15
        assert d["stages"] == int(name.split("_p")[1].split("_")[0])
        assert d["schedule"] == (pt.PT_SCHED_STREAMK if name.endswith("_stk") else pt.PT_SCHED_PERSISTENT)


@pytest.mark.parametrize("name", PAIRS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (100, 70, 64), (129, 130, 300), (256, 128, 64), (300, 200, 600),
                                   (520, 257, 129), (384, 64, 1000)])
def test_pair_small_integers_bit_exact(name, shape):
    M, N, K = shape
    A = matrix("ints", 31, M, K)
    B = matrix("ints", 32, K, N)
    ref = og.gemm(A, B)
    out = _run(name, A, B, M, N)
    assert np.array_equal(out.astype(np.float64), ref), (name, shape)


@pytest.mark.parametrize("name", PAIRS)
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_pair_every_plane_bit_exact(name, ta, tb):
    # entries that need every plane of the split; exact integer result
    M, N, K = 300, 200, 520
    A, B, _ = wide_int_operands(17, M, N, K)
    As = A.T if ta == "T" else A
    Bs = B.T if tb == "T" else B
    ref = og.gemm(A, B)
    out = _run(name, As, Bs, M, N, ta, tb)
    assert np.array_equal(out.astype(np.float64), ref), (name, ta, tb)


@pytest.mark.parametrize("name", PAIRS)
def test_pair_more_tiles_than_pairs(name):
    # 16 x 8 = 128 pair tiles on at most 76 resident pairs; sampled rows vs the oracle
    M, N, K = 4096, 1024, 1024
    A = matrix("uniform", 41, M, K)
    B = matrix("uniform", 42, K, N)
    out = _run(name, A, B, M, N)
    rows = np.random.default_rng(5).choice(M, 64, replace=False)
    rows = np.concatenate([rows, [0, 127, 128, 255, 256, M - 1]])
    ref = og.gemm(A[rows], B)
    err = np.abs(out[rows].astype(np.float64) - ref).max() / K
    assert err <= 2e-6, (name, err)
    assert pt.device_status() == 0


@pytest.mark.parametrize("name", PAIRS)
def test_pair_alpha_beta(name):
    M, N, K = 300, 200, 1000
    A = matrix("uniform", 61, M, K)
    B = matrix("uniform", 62, K, N)
    C0 = matrix("uniform", 63, M, N)
    ref = og.gemm(A, B, alpha=0.75, beta=-1.5, C=C0)
    out = _run(name, A, B, M, N, alpha=0.75, beta=-1.5, C0=C0)
    assert np.abs(out - ref).max() <= 2e-6 * (K * 0.75 + 1.5), name
    assert pt.device_status() == 0


@pytest.mark.parametrize("name", ["tc3xf16_m256n256_p6_sw64_2sm", "tc3xf16_m256n256_p5_sw64_2sm"])
def test_pair_hybrid_streamk_tail(name):
    # 10 x 10 = 100 pair tiles: more than the resident pairs, with a last wave
    # under 3/4 full, so the hybrid runs its stream-K pair instantiation;
    # repeated launches must not read earlier launches' partial tiles.
    M, N, K = 2560, 2560, 1024
    A, B, _ = wide_int_operands(19, M, N, K)
    ref = og.gemm(A, B)
    for _ in range(3):
        out = _run(name, A, B, M, N)
        assert np.array_equal(out.astype(np.float64), ref), name
    assert pt.device_status() == 0
