"""The allocation-free SGEMM entry point (pt_sgemm_3xtf32_noalloc).

Callers that cannot allocate device memory during their GEMM calls use this
entry point; it keeps its split planes in a fixed array inside the library.
This test calls it through the C ABI, twice in a row with different shapes
and layouts, and checks each result against the existing entry point running
the same 3xTF32 variant, within the normalised-error bound the other tests
use.  It also checks that a shape too large for the array is refused.
"""

import ctypes

import numpy as np
import pytest

from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")
from paper_2507_15277_gb300 import _lib  # noqa: E402


def _noalloc(A, B, C, ta, tb, alpha, beta, stream):
    lib = _lib.lib()
    M, N = C.shape
    K = A.shape[1] if ta == "N" else A.shape[0]
    return lib.pt_sgemm_3xtf32_noalloc(
        ta.encode(), tb.encode(), M, N, K, alpha, ctypes.c_void_p(A.data_ptr()), A.stride(0),
        ctypes.c_void_p(B.data_ptr()), B.stride(0), beta, ctypes.c_void_p(C.data_ptr()), C.stride(0),
        ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_existing_entry_point_twice():
    vid = pt.variant_by_name("tc3xtf32_m128n128_p3")
    stream = torch.cuda.current_stream()
    cases = [(1000, 700, 900, "N", "N", 1.0, 0.0, 11), (513, 1100, 257, "T", "T", 1.5, -0.5, 12)]
    for (M, N, K, ta, tb, alpha, beta, seed) in cases:
        A = matrix("uniform", seed, M, K)
        B = matrix("uniform", seed + 100, K, N)
        C0 = matrix("uniform", seed + 200, M, N)
        Ad = torch.from_numpy(np.ascontiguousarray(A.T if ta == "T" else A)).cuda()
        Bd = torch.from_numpy(np.ascontiguousarray(B.T if tb == "T" else B)).cuda()
        want = torch.from_numpy(C0).cuda()
        got = torch.from_numpy(C0).cuda()
        pt.sgemm(Ad, Bd, want, ta, tb, alpha, beta, variant=vid)
        rc = _noalloc(Ad, Bd, got, ta, tb, alpha, beta, stream)
        assert rc == 0, _lib.lib().pt_last_error()
        torch.cuda.synchronize()
        err = normalised_error(got.cpu().numpy(), want.cpu().numpy(), K, np.abs(A).max(), np.abs(B).max(),
                               alpha, beta, np.abs(C0).max())
        assert err <= TOL_FP32, (M, N, K, err)


def test_noalloc_refuses_shapes_beyond_its_array():
    stream = torch.cuda.current_stream()
    M = N = K = 4096  # 2 * 8192 * 4096 * 4 bytes = 256 MiB > 64 MiB
    A = torch.zeros((1, 1), device="cuda")
    C = torch.zeros((1, 1), device="cuda")
    lib = _lib.lib()
    rc = lib.pt_sgemm_3xtf32_noalloc(b"N", b"N", M, N, K, 1.0, ctypes.c_void_p(A.data_ptr()), K,
                                     ctypes.c_void_p(A.data_ptr()), N, 0.0, ctypes.c_void_p(C.data_ptr()), N,
                                     ctypes.c_void_p(stream.cuda_stream))
    assert rc == _lib.PT_EINVAL
    assert b"scratch" in lib.pt_last_error()
