"""The allocation-free SGEMM entry point (pt_sgemm_3xtf32_noalloc).

Some callers cannot allocate device memory while they run GEMMs: programs
that hand all device memory to their own pool allocator at start-up,
latency-critical loops where an allocation may synchronise the device, and
hosts that only run with memory reserved in advance.  This entry point keeps
its split planes in a fixed array inside the library instead of a workspace.

The test calls it through the C ABI, several times in a row with different
shapes, layouts and scalars, and checks each result
  * against the FP64 CPU oracle, within the normalised-error bound 2e-6 that
    the other parity tests use, and
  * bit for bit against the registry's tc3xtf32_m128n128_p3 (the same split,
    the same kernel, the same per-tile MMA order) run through pt_sgemm_variant.
It covers the quick-return paths (K = 0, alpha = 0), an A whose rows are not
16-byte aligned (odd lda, and a 4-byte offset pointer), and checks that free
device memory does not change across a call after the first one, and that a
shape too large for the array is refused.

This file is collected last, and passes alone in a fresh process as well as
after the other tests.
"""

import ctypes

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")
from paper_2507_15277_gb300 import _lib  # noqa: E402

DEV = "cuda:0"


def _noalloc(A, B, C, ta, tb, alpha, beta, M, N, K, lda, ldb, stream):
    lib = _lib.lib()
    return lib.pt_sgemm_3xtf32_noalloc(
        ta.encode(), tb.encode(), M, N, K, alpha, ctypes.c_void_p(A.data_ptr()), lda,
        ctypes.c_void_p(B.data_ptr()), ldb, beta, ctypes.c_void_p(C.data_ptr()), C.stride(0),
        ctypes.c_void_p(stream.cuda_stream))


def _storage(X, t, ld, offset):
    """Row-major storage of op^-1(X) with leading dimension ld, starting
    `offset` floats into a device buffer (NaN everywhere else)."""
    S = np.ascontiguousarray(X.T if t == "T" else X)
    rows, cols = S.shape
    buf = np.full(offset + rows * ld, np.nan, np.float32)
    view = buf[offset:].reshape(rows, ld)
    view[:, :cols] = S
    d = torch.from_numpy(buf).to(DEV)
    return d[offset:], S, view


# (M, N, K, transA, transB, alpha, beta, seed, lda pad, A offset in floats)
CASES = [
    (1000, 700, 900, "N", "N", 1.0, 0.0, 11, 0, 0),
    (513, 1100, 257, "T", "T", 1.5, -0.5, 12, 0, 0),
    (300, 260, 1000, "N", "T", 1.0, 0.0, 13, 1, 0),   # odd lda: unaligned rows of A
    (257, 384, 520, "N", "N", -2.0, 1.0, 14, 0, 1),   # A starts 4 bytes off alignment
    (200, 136, 64, "T", "N", 0.0, 2.0, 15, 0, 0),     # alpha = 0: C <- 2 C
    (96, 80, 0, "N", "N", 1.0, 2.0, 16, 0, 0),        # K = 0: C <- 2 C
]


def _run_case(M, N, K, ta, tb, alpha, beta, seed, pad, off, stream):
    A = matrix("uniform", seed, M, K)
    B = matrix("uniform", seed + 100, K, N)
    C0 = matrix("uniform", seed + 200, M, N)
    lda = (K if ta == "N" else M) + pad
    ldb = N if tb == "N" else K
    Ad, As, Av = _storage(A, ta, max(lda, 1), off)
    Bd, Bs, Bv = _storage(B, tb, max(ldb, 1), 0)
    got = torch.from_numpy(C0).to(DEV)
    rc = _noalloc(Ad, Bd, got, ta, tb, alpha, beta, M, N, K, max(lda, 1), max(ldb, 1), stream)
    assert rc == 0, _lib.lib().pt_last_error()
    torch.cuda.synchronize()
    out = got.cpu().numpy()
    ref = og.gemm(Av, Bv, ta, tb, alpha=alpha, beta=beta, C=C0, M=M, N=N, K=K)
    err = normalised_error(out, ref, K, np.abs(A).max() if K else 0.0, np.abs(B).max() if K else 0.0,
                           alpha, beta, np.abs(C0).max())
    assert err <= TOL_FP32, (M, N, K, ta, tb, err)
    if K and alpha != 0.0:
        # the registry's twin: same planes, same kernel, same bits
        Al = Ad.as_strided((As.shape[0], As.shape[1]), (max(lda, 1), 1))
        Bl = Bd.as_strided((Bs.shape[0], Bs.shape[1]), (max(ldb, 1), 1))
        twin = torch.from_numpy(C0).to(DEV)
        pt.sgemm(Al, Bl, twin, ta, tb, alpha, beta, variant=pt.variant_by_name("tc3xtf32_m128n128_p3"))
        torch.cuda.synchronize()
        assert np.array_equal(out.view(np.uint32), twin.cpu().numpy().view(np.uint32)), (M, N, K, ta, tb)
    else:
        assert np.array_equal(out.astype(np.float64), ref)  # beta * C is one rounding: exact here


def test_noalloc_matches_oracle_and_twin_on_consecutive_calls():
    stream = torch.cuda.current_stream()
    for case in CASES:
        _run_case(*case, stream=stream)
    for case in CASES[:2]:  # again: the array keeps the last call's planes
        _run_case(*case, stream=stream)
    assert pt.device_status() == 0


def test_noalloc_second_call_allocates_nothing():
    stream = torch.cuda.current_stream()
    M, N, K = 640, 512, 768
    A = torch.from_numpy(matrix("uniform", 21, M, K)).to(DEV)
    B = torch.from_numpy(matrix("uniform", 22, K, N)).to(DEV)
    C = torch.empty((M, N), device=DEV)
    assert _noalloc(A, B, C, "N", "N", 1.0, 0.0, M, N, K, K, N, stream) == 0   # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(A, B, C, "N", "N", 1.0, 0.0, M, N, K, K, N, stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_refuses_shapes_beyond_its_array():
    stream = torch.cuda.current_stream()
    M = N = K = 4096  # 2 * 8192 * 4096 * 4 bytes = 256 MiB > 64 MiB
    A = torch.zeros((1, 1), device=DEV)
    C = torch.zeros((1, 1), device=DEV)
    lib = _lib.lib()
    rc = lib.pt_sgemm_3xtf32_noalloc(b"N", b"N", M, N, K, 1.0, ctypes.c_void_p(A.data_ptr()), K,
                                     ctypes.c_void_p(A.data_ptr()), N, 0.0, ctypes.c_void_p(C.data_ptr()), N,
                                     ctypes.c_void_p(stream.cuda_stream))
    assert rc == _lib.PT_EINVAL
    assert b"scratch" in lib.pt_last_error()
