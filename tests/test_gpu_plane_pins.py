"""GPU: bit-exact pins that reach every plane of the split-precision versions.

The small-integer parity tests use entries in [-8, 8], which are exact in a
single BF16 or TF32 plane, so they cannot see a wrong or missing residual
product.  These pins use inputs whose exact product is an integer below 2^24
in every partial sum (so every summation order in FP32 gives the exact
result) and whose entries need two or three planes:

* rank-1 closed form: a_ik = 1, b_kj = k, so C_ij = K(K-1)/2 for every
  (i, j); for K > 256 the b_kj need two BF16 planes, for K > 2048 two TF32
  planes;
* wide integers (workloads.wide_int_operands): 18-bit, 9-bit and +-1
  entries arranged so that every product the BF16x3 split keeps (b_i b_j,
  i + j <= 2) and every one the 3xTF32 split keeps (hi hi, hi lo, lo hi) is
  non-zero for many outputs, and every product they drop is zero; the same
  holds for the scaled 3xF16 split (h0 h0, h0 h1, h1 h0), whose per-chunk
  power-of-two scales change no significand bit (the CPU tests in
  test_split_planes.py establish these facts).

Every registered variant -- FP32 SIMT (with and without cluster split-K),
3xTF32, BF16x3 and 3xF16 in every schedule (persistent, stream-K, cluster
split-K 2/4/8), with fused A or B splitting and 32-column tiles -- must reproduce the
FP64 oracle's result bit for bit.  The operation is the paper's GEMM
(Section V-B); the split is an extension of the variant family.
"""

import numpy as np
import pytest

from oracle import gemm as og
from workloads import rank1_operands, wide_int_operands

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
_cache = {}


def _layout_ok(desc, ta, tb):
    return bool(desc["trans_mask"] >> ((ta == "T") * 2 + (tb == "T")) & 1)


def _case(name, M, N, K, ta, tb):
    """Device storage of op^-1(A), op^-1(B) and the oracle's exact result."""
    key = (name, M, N, K, ta, tb)
    if key not in _cache:
        if name == "rank1":
            A, B = rank1_operands(M, N, K)
        else:
            A, B, _ = wide_int_operands(17, M, N, K)
        As = np.ascontiguousarray(A.T if ta == "T" else A)
        Bs = np.ascontiguousarray(B.T if tb == "T" else B)
        ref = og.gemm(As, Bs, ta, tb, M=M, N=N, K=K)
        if name == "rank1":
            assert np.all(ref == K * (K - 1) / 2)
        _cache[key] = (torch.from_numpy(As).to(DEV), torch.from_numpy(Bs).to(DEV), ref)
    return _cache[key]


# (input set, M, N, K): several tiles in M and N with ragged edges; K spans
# one 128-k chunk, several chunks, a ragged chunk and 32 chunks (split-K,
# stream-K hand-over of partial tiles).
CASES = [("rank1", 200, 136, 128), ("rank1", 200, 136, 1024), ("rank1", 300, 136, 4096),
         ("wide", 300, 200, 1024), ("wide", 300, 136, 4096), ("wide", 260, 72, 1000)]


def _nvar():
    return pt.num_variants()


@pytest.mark.parametrize("vid", range(456))
def test_every_plane_bit_exact(vid):
    if vid >= _nvar():
        pytest.skip("registry has fewer variants")
    d = pt.variant(vid)
    ran = 0
    for (name, M, N, K) in CASES:
        layouts = [("N", "N"), ("T", "T"), ("N", "T"), ("T", "N")]
        if K == 1000:
            layouts = layouts[1:] + layouts[:1]     # a transposed layout first
        for ta, tb in layouts:
            if _layout_ok(d, ta, tb):
                break
        else:
            continue
        Ad, Bd, ref = _case(name, M, N, K, ta, tb)
        C = torch.full((M, N), float("nan"), device=DEV)
        try:
            pt.sgemm(Ad, Bd, C, ta, tb, variant=vid)
        except pt.PtError as e:
            assert e.code == pt._lib.PT_EUNSUPPORTED, (d["name"], name, M, N, K)
            continue
        torch.cuda.synchronize()
        out = C.cpu().numpy().astype(np.float64)
        bad = np.argwhere(out != ref)
        assert bad.size == 0, (d["name"], name, (M, N, K, ta, tb), len(bad), bad[:3].tolist(),
                               [(out[i, j], ref[i, j]) for i, j in bad[:3]])
        ran += 1
    assert ran >= 3, (d["name"], ran)
    assert pt.device_status() == 0


def test_selector_entry_every_plane():
    """pt_sgemm with no manifest loaded (the default variant): exact too."""
    for (name, M, N, K) in CASES:
        Ad, Bd, ref = _case(name, M, N, K, "N", "N")
        C = pt.sgemm(Ad, Bd)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.float64), ref), (name, M, N, K)
