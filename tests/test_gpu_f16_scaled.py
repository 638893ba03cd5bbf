"""GPU: the scaled 3xF16 tensor-core versions on inputs whose magnitudes
differ by row, by column and along k.

Per 256 values of k, each row of op(A) and each group of 32 consecutive
columns of op(B) is scaled by a power of two before the FP16 split, so the
error of C_ij is bounded by the magnitudes in row i of A and in the 32-column
group of j in B, not by the largest entries of the matrices.  The test holds
every entry to that per-entry form of the bound,
  |C_ij - C_ref_ij| <= 2e-6 * K * max_k |A_ik| * max_{k, j' in group(j)} |B_kj'|,
against the FP64 oracle, on every 3xF16 version, with row and column scales
spread over 2^-30 .. 2^27, magnitudes changing along k, and both ends of
the supported range (maxima 2^-45 and 2^70).
"""

import numpy as np
import pytest

from oracle import gemm as og
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"


def _f16_variants():
    return [v for v in pt.variants() if v["kind"] == 3]


def _scaled_case(M, N, K, seed):
    A = matrix("uniform", seed, M, K).astype(np.float64)
    B = matrix("uniform", seed + 1, K, N).astype(np.float64)
    A *= np.ldexp(1.0, 3 * (np.arange(M) % 20) - 30)[:, None]          # rows: 2^-30 .. 2^27
    B *= np.ldexp(1.0, 2 * (np.arange(N) % 15) - 15)[None, :]          # columns: 2^-15 .. 2^13
    A *= np.ldexp(1.0, 5 * (np.arange(K) // 128 % 4) - 8)[None, :]    # chunks of k: 2^-8 .. 2^7
    return A.astype(np.float32), B.astype(np.float32)


def _check_entrywise(C, ref, A, B, K, name):
    ra = np.abs(A.astype(np.float64)).max(axis=1)[:, None]
    colmax = np.abs(B.astype(np.float64)).max(axis=0)
    N = colmax.size
    groups = np.pad(colmax, (0, -N % 32)).reshape(-1, 32).max(axis=1)
    cb = np.repeat(groups, 32)[:N][None, :]   # the largest |B| of j's 32-column group
    bound = 2e-6 * K * ra * cb
    err = np.abs(C.astype(np.float64) - ref)
    worst = float((err / bound).max())
    assert np.all(np.isfinite(C)) and worst <= 1.0, (name, worst)
    return worst


def test_f16_versions_exist():
    names = {v["name"] for v in _f16_variants()}
    assert {"tc3xf16_m128n128_p3", "tc3xf16_m128n128_p3_stk", "tc3xf16_m128n64_p4_sk8"} <= names


@pytest.mark.parametrize("shape", [(300, 200, 1000), (640, 384, 2176), (128, 256, 4096)])
def test_f16_entrywise_bound_with_row_column_and_chunk_scales(shape):
    M, N, K = shape
    A, B = _scaled_case(M, N, K, 41)
    ref = og.gemm(A, B)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    for v in _f16_variants():
        C = torch.full((M, N), float("nan"), device=DEV)
        pt.sgemm(Ad, Bd, C, variant=v["id"])
        torch.cuda.synchronize()
        _check_entrywise(C.cpu().numpy(), ref, A, B, K, v["name"])
    # the other kinds, whose error is relative to each product, meet it too
    for name in ("tc3xtf32_m128n128_p3", "tcbf16x3_m128n128_p2"):
        C = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(name))
        torch.cuda.synchronize()
        _check_entrywise(C.cpu().numpy(), ref, A, B, K, name)
    assert pt.device_status() == 0


@pytest.mark.parametrize("ta,tb", [("T", "T"), ("N", "T"), ("T", "N")])
def test_f16_transposed_layouts(ta, tb):
    M, N, K = 260, 136, 700
    A, B = _scaled_case(M, N, K, 43)
    ref = og.gemm(A, B)
    As = np.ascontiguousarray(A.T if ta == "T" else A)
    Bs = np.ascontiguousarray(B.T if tb == "T" else B)
    Ad, Bd = torch.from_numpy(As).to(DEV), torch.from_numpy(Bs).to(DEV)
    for v in _f16_variants():
        C = pt.sgemm(Ad, Bd, transA=ta, transB=tb, variant=v["id"])
        torch.cuda.synchronize()
        _check_entrywise(C.cpu().numpy(), ref, A, B, K, (v["name"], ta, tb))


@pytest.mark.parametrize("ea,eb", [(70, -45), (-45, 70), (-40, -40)])
def test_f16_ends_of_the_supported_range(ea, eb):
    # every value of A near 2^ea and of B near 2^eb
    M, N, K = 200, 136, 520
    A = (matrix("uniform", 51, M, K).astype(np.float64) * 2.0 ** ea).astype(np.float32)
    B = (matrix("uniform", 52, K, N).astype(np.float64) * 2.0 ** eb).astype(np.float32)
    ref = og.gemm(A, B)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    for name in ("tc3xf16_m128n128_p3", "tc3xf16_m128n64_p4_sk4", "tc3xf16_m128n128_p6_sw64_stk"):
        C = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(name))
        torch.cuda.synchronize()
        _check_entrywise(C.cpu().numpy(), ref, A, B, K, (name, ea, eb))


def test_f16_alpha_beta_and_beta_zero_ignores_c():
    M, N, K = 300, 200, 1000
    A = matrix("uniform", 61, M, K)
    B = matrix("uniform", 62, K, N)
    C0 = matrix("uniform", 63, M, N)
    ref = og.gemm(A, B, alpha=0.75, beta=-1.5, C=C0)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    bound = 2e-6 * (K * 0.75 + 1.5)
    for v in _f16_variants():
        C = torch.from_numpy(C0).to(DEV)
        pt.sgemm(Ad, Bd, C, alpha=0.75, beta=-1.5, variant=v["id"])
        Cz = torch.full((M, N), float("nan"), device=DEV)
        pt.sgemm(Ad, Bd, Cz, variant=v["id"])
        torch.cuda.synchronize()
        assert np.abs(C.cpu().numpy() - ref).max() <= bound, v["name"]
        assert np.all(np.isfinite(Cz.cpu().numpy())), v["name"]
