"""GPU: tensor-core versions that split B (or A) inside the GEMM kernel
(converter warps write the BF16 planes into shared memory).  They must give
exactly the bits of the version that splits both operands in the split
kernel (same planes, same MMA order), stay within the FP32 bound against the
oracle, handle ragged edges, and decline layouts they cannot read."""

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
PAIRS = [("tcbf16x3_m128n64_p2_fb", "tcbf16x3_m128n64_p2"),
         ("tcbf16x3_m128n64_p2_fb_sk2", "tcbf16x3_m128n64_p2"),
         ("tcbf16x3_m128n64_p2_fb_sk4", "tcbf16x3_m128n64_p2_sk4"),
         ("tcbf16x3_m128n64_p2_fb_stk", "tcbf16x3_m128n64_p2"),
         # 64-byte rows: the twin with the same rows, tile and chunk order
         ("tcbf16x3_m128n64_p5_sw64_fb", "tcbf16x3_m128n64_p4_sw64"),
         ("tcbf16x3_m128n128_p3_sw64_fb", "tcbf16x3_m128n128_p4_sw64"),
         ("tcbf16x3_m128n128_p3_sw64_fb_sk4", "tcbf16x3_m128n128_p4_sw64_sk4"),
         ("tcbf16x3_m128n128_p3_sw64_fb_stk", "tcbf16x3_m128n128_p4_sw64")]
SHAPES = [(128, 4096, 4096), (128, 1000, 1000), (300, 200, 520), (640, 320, 2176)]


@pytest.mark.parametrize("fused,plain", PAIRS)
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_b_matches_split_kernel_and_oracle(fused, plain, shape):
    M, N, K = shape
    A = matrix("uniform", 31, M, K)
    B = matrix("uniform", 32, K, N)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    Cf = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(fused))
    Cp = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(plain))
    torch.cuda.synchronize()
    cf = Cf.cpu().numpy()
    if "_sk" not in fused and "_stk" not in fused and "_sk" not in plain:
        assert np.array_equal(cf, Cp.cpu().numpy())  # identical planes and products
    rows = np.arange(0, M, max(1, M // 64))
    ref = og.gemm(A, B, rows=rows)
    assert normalised_error(cf[rows], ref, K, np.abs(A).max(), np.abs(B).max()) <= TOL_FP32
    assert pt.device_status() == 0


@pytest.mark.parametrize("fused", [p[0] for p in PAIRS])
def test_fused_b_integers_transposed_a_and_alpha_beta(fused):
    M, N, K = 200, 136, 1032
    A = matrix("ints", 41, K, M)          # stored K x M: transA = 'T'
    B = matrix("ints", 42, K, N)
    C0 = matrix("ints", 43, M, N)
    ref = og.gemm(A, B, "T", "N", alpha=2.0, beta=-1.0, C=C0, M=M, N=N, K=K)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.from_numpy(C0.copy()).to(DEV)
    pt.sgemm(Ad, Bd, C, transA="T", alpha=2.0, beta=-1.0, variant=pt.variant_by_name(fused))
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)


def test_fused_b_declines_unreadable_b():
    vid = pt.variant_by_name("tcbf16x3_m128n64_p2_fb")
    A = torch.ones((128, 64), device=DEV)
    Bt = torch.ones((96, 64), device=DEV)          # transB = 'T': B stored N x K
    with pytest.raises(pt.PtError) as e:
        pt.sgemm(A, Bt, transB="T", variant=vid)
    assert e.value.code == pt._lib.PT_EUNSUPPORTED
    Bs = torch.ones((64, 99), device=DEV)[:, :97]   # ldb = 99: rows not 16-byte aligned
    with pytest.raises(pt.PtError) as e:
        pt.sgemm(A, Bs, variant=vid)
    assert e.value.code == pt._lib.PT_EUNSUPPORTED
    # The runtime selector never needs them: pt_sgemm still runs these layouts.
    C = pt.sgemm(A, Bt, transB="T")
    torch.cuda.synchronize()
    assert torch.all(C == 64.0)


PAIRS_A = [("tcbf16x3_m128n64_p3_sw64_fa", "tcbf16x3_m128n64_p4_sw64"),
           ("tcbf16x3_m128n64_p3_sw64_fa_sk2", "tcbf16x3_m128n64_p4_sw64"),
           ("tcbf16x3_m128n64_p3_sw64_fa_sk4", "tcbf16x3_m128n64_p4_sw64_sk4"),
           ("tcbf16x3_m128n64_p3_sw64_fa_stk", "tcbf16x3_m128n64_p4_sw64"),
           ("tcbf16x3_m128n64_p4_sw64_fa", "tcbf16x3_m128n64_p4_sw64"),
           ("tcbf16x3_m128n128_p3_sw64_fa", "tcbf16x3_m128n128_p4_sw64"),
           ("tcbf16x3_m128n128_p3_sw64_fa_sk4", "tcbf16x3_m128n128_p4_sw64_sk4"),
           ("tcbf16x3_m128n128_p3_sw64_fa_stk", "tcbf16x3_m128n128_p4_sw64")]
SHAPES_A = [(4096, 128, 4096), (1000, 128, 1000), (300, 200, 520), (640, 320, 2176)]


@pytest.mark.parametrize("fused,plain", PAIRS_A)
@pytest.mark.parametrize("shape", SHAPES_A)
def test_fused_a_matches_split_kernel_and_oracle(fused, plain, shape):
    M, N, K = shape
    A = matrix("uniform", 51, M, K)
    B = matrix("uniform", 52, K, N)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    Cf = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(fused))
    Cp = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(plain))
    torch.cuda.synchronize()
    cf = Cf.cpu().numpy()
    if "_sk" not in fused and "_stk" not in fused:
        # same planes and the same k-chunk order (stage depth does not change the arithmetic)
        assert np.array_equal(cf, Cp.cpu().numpy())
    rows = np.arange(0, M, max(1, M // 64))
    ref = og.gemm(A, B, rows=rows)
    assert normalised_error(cf[rows], ref, K, np.abs(A).max(), np.abs(B).max()) <= TOL_FP32
    assert pt.device_status() == 0


@pytest.mark.parametrize("fused", [p[0] for p in PAIRS_A])
def test_fused_a_integers_transposed_b_and_alpha_beta(fused):
    M, N, K = 200, 136, 1032
    A = matrix("ints", 61, M, K)
    B = matrix("ints", 62, N, K)          # stored N x K: transB = 'T'
    C0 = matrix("ints", 63, M, N)
    ref = og.gemm(A, B, "N", "T", alpha=2.0, beta=-1.0, C=C0, M=M, N=N, K=K)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.from_numpy(C0.copy()).to(DEV)
    pt.sgemm(Ad, Bd, C, transB="T", alpha=2.0, beta=-1.0, variant=pt.variant_by_name(fused))
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)


def test_fused_a_declines_unreadable_a():
    vid = pt.variant_by_name("tcbf16x3_m128n64_p3_sw64_fa")
    At = torch.ones((64, 128), device=DEV)          # transA = 'T': A stored K x M
    B = torch.ones((64, 96), device=DEV)
    with pytest.raises(pt.PtError) as e:
        pt.sgemm(At, B, transA="T", variant=vid)
    assert e.value.code == pt._lib.PT_EUNSUPPORTED


PAIRS_AB = [("tcbf16x3_m128n64_p3_sw64_fab", "tcbf16x3_m128n64_p4_sw64"),
            ("tcbf16x3_m128n64_p3_sw64_fab_sk2", "tcbf16x3_m128n64_p4_sw64_sk2"),
            ("tcbf16x3_m128n64_p3_sw64_fab_sk4", "tcbf16x3_m128n64_p4_sw64_sk4"),
            ("tcbf16x3_m128n128_p2_sw64_fab", "tcbf16x3_m128n128_p4_sw64"),
            ("tcbf16x3_m128n128_p2_sw64_fab_sk4", "tcbf16x3_m128n128_p4_sw64_sk4")]
SHAPES_AB = [(128, 128, 128), (300, 200, 520), (640, 320, 2176), (1024, 1024, 512), (128, 128, 4096)]


@pytest.mark.parametrize("fused,plain", PAIRS_AB)
@pytest.mark.parametrize("shape", SHAPES_AB)
def test_fused_both_matches_split_kernel_and_oracle(fused, plain, shape):
    # Both operands split inside the GEMM kernel (one launch): the same planes
    # and the same chunk order (and split-K slices) as the twin that splits
    # both in the split kernel, so the same bits.
    M, N, K = shape
    A = matrix("uniform", 71, M, K)
    B = matrix("uniform", 72, K, N)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    Cf = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(fused))
    Cp = pt.sgemm(Ad, Bd, variant=pt.variant_by_name(plain))
    torch.cuda.synchronize()
    cf = Cf.cpu().numpy()
    assert np.array_equal(cf, Cp.cpu().numpy())
    rows = np.arange(0, M, max(1, M // 64))
    ref = og.gemm(A, B, rows=rows)
    assert normalised_error(cf[rows], ref, K, np.abs(A).max(), np.abs(B).max()) <= TOL_FP32
    assert pt.device_status() == 0


@pytest.mark.parametrize("fused", [p[0] for p in PAIRS_AB])
def test_fused_both_integers_alpha_beta_and_declines(fused):
    M, N, K = 200, 136, 1032
    A = matrix("ints", 81, M, K)
    B = matrix("ints", 82, K, N)
    C0 = matrix("ints", 83, M, N)
    ref = og.gemm(A, B, alpha=2.0, beta=-1.0, C=C0)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.from_numpy(C0.copy()).to(DEV)
    vid = pt.variant_by_name(fused)
    pt.sgemm(Ad, Bd, C, alpha=2.0, beta=-1.0, variant=vid)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
    for ta, tb in (("T", "N"), ("N", "T")):     # only A as M x K and B as K x N are read in the kernel
        At = Ad if ta == "N" else Ad.t().contiguous()
        Bt = Bd if tb == "N" else Bd.t().contiguous()
        with pytest.raises(pt.PtError) as e:
            pt.sgemm(At, Bt, transA=ta, transB=tb, variant=vid)
        assert e.value.code == pt._lib.PT_EUNSUPPORTED
