"""GPU: sizes at the edges of what the path handles.  Very long K (2^18:
the tensor-core versions restart their accumulator 2048 times and promote
every chunk), very tall and very wide operands (grids of tens of thousands of
tiles, split grids of thousands of rows), and degenerate extents (M, N or K
of 1).  Results are checked against the FP64 oracle on sampled rows."""

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
VARIANTS = [None, "s128x128x8_w32x64_t8x8_kl1_v1_p2_sk1_cpm", "tcbf16x3_m128n128_p4_sw64_stk",
            "tcbf16x3_m128n64_p3_sk8", "tc3xtf32_m128n128_p3", "tcbf16x3_m128n64_p2_fb_sk4",
            "tcbf16x3_m128n128_p3_sw64_fa_sk4", "tcbf16x3_m128n128_p3_sw64_fb_stk"]


def _check(M, N, K, name, kind="uniform", rows=16):
    A = matrix(kind, 91, M, K)
    B = matrix(kind, 92, K, N)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    vid = None if name is None else pt.variant_by_name(name)
    C = pt.sgemm(Ad, Bd, variant=vid)
    torch.cuda.synchronize()
    r = np.unique(np.linspace(0, M - 1, min(rows, M)).astype(np.int64))
    ref = og.gemm(A, B, rows=r)
    e = normalised_error(C[r].cpu().numpy(), ref, K, np.abs(A).max(), np.abs(B).max())
    assert e <= TOL_FP32, (M, N, K, name, e)
    assert pt.device_status() == 0


@pytest.mark.parametrize("name", VARIANTS)
def test_very_long_k(name):
    _check(128, 128, 1 << 18, name)


@pytest.mark.parametrize("name", VARIANTS)
def test_very_tall_a(name):
    _check(1 << 17, 128, 64, name)


@pytest.mark.parametrize("name", VARIANTS)
def test_very_wide_b(name):
    _check(128, 1 << 17, 64, name)


@pytest.mark.parametrize("name", VARIANTS)
@pytest.mark.parametrize("shape", [(1, 257, 33), (257, 1, 33), (65, 70, 1), (1, 1, 4097)])
def test_degenerate_extents_exact(name, shape):
    M, N, K = shape
    A = matrix("ints", 93, M, K)
    B = matrix("ints", 94, K, N)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    vid = None if name is None else pt.variant_by_name(name)
    try:
        C = pt.sgemm(Ad, Bd, variant=vid)
    except pt.PtError as e:  # a variant's admission rules may refuse (e.g. alignment of a 1-wide B)
        assert e.code == pt._lib.PT_EUNSUPPORTED
        return
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.float64), og.gemm(A, B, M=M, N=N, K=K))
