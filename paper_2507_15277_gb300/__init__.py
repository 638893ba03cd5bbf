"""Portability-tuned FP32 GEMM for GB300 (sm_103a): Python face of libptsgemm.

Every function here only marshals arguments into the C ABI declared in
``include/pt_sgemm.h``; all GEMM work runs in the library's CUDA kernels and
all tuning/selection arithmetic in its C++ code.  PyTorch supplies device
memory and streams.

    import paper_2507_15277_gb300 as pt
    C = pt.sgemm(A, B)                       # multi-versioned entry (runtime selector)
    C = pt.sgemm(A, B, variant=17)           # one specific variant
    pt.tune(shapes, "table.csv")             # timing table (Section V-D)
    ids, g = pt.select("table.csv", train, k=4, manifest="kappa.json")   # PortabilityTune
    pt.load_manifest("kappa.json")           # install kappa for pt.sgemm
"""

from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (PT_LOADER_CPASYNC, PT_LOADER_TMA, PT_SCHED_PERSISTENT,  # noqa: F401
                   PT_SCHED_STREAMK, PT_SCHED_TILE, PT_SCORE_BEST_OF_SET, PT_SCORE_SELECTOR, PT_SELECT_AUTO,
                   PT_SELECT_EXACT, PT_SELECT_GREEDY_SWAP, PT_SELECT_KMEANS, PT_SELECT_TREE, PtError, Shape,
                   TuneOpts, VariantDesc)

__all__ = [
    "sgemm", "reference", "num_variants", "variant", "variants", "variant_by_name", "default_variant",
    "tune", "select", "score", "table_shapes", "load_manifest", "selected_variant", "device_status",
    "grouped_problems", "upload_problems", "sgemm_grouped", "kernel_timer_start", "kernel_timer_stop", "shutdown",
    "PtError",
]


def _l():
    return _lib.lib()


def num_variants() -> int:
    return _l().pt_num_variants()


def variant(i: int) -> dict:
    d = VariantDesc()
    _lib.check(_l().pt_variant_desc(int(i), ctypes.byref(d)), "pt_variant_desc")
    return d.as_dict()


def variants() -> list:
    return [variant(i) for i in range(num_variants())]


def variant_by_name(name: str) -> int:
    return _lib.check(_l().pt_variant_by_name(name.encode()), "pt_variant_by_name")


def default_variant() -> int:
    return _l().pt_default_variant()


# ---- GEMM ---------------------------------------------------------------------------
def _dims(A, B, transA, transB):
    if A.dim() != 2 or B.dim() != 2:
        raise ValueError("A and B must be 2-D")
    M, KA = (A.shape[0], A.shape[1]) if transA == "N" else (A.shape[1], A.shape[0])
    KB, N = (B.shape[0], B.shape[1]) if transB == "N" else (B.shape[1], B.shape[0])
    if KA != KB:
        raise ValueError("inner dimensions differ: %d vs %d" % (KA, KB))
    return M, N, KA


def _ld(t):
    import torch
    if t.dtype != torch.float32:
        raise TypeError("float32 tensors only")
    if t.numel() == 0:
        return max(int(t.shape[1]), 1)
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("row-major storage with unit column stride required")
    return max(int(t.stride(0)), int(t.shape[1]), 1) if t.shape[0] > 1 else max(int(t.shape[1]), 1)


def _stream(stream, device):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _call(fn, where, A, B, C, transA, transB, alpha, beta, stream, pre=()):
    import torch
    M, N, K = _dims(A, B, transA, transB)
    for t, n in ((A, "A"), (B, "B"), (C, "C")):
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % n)
    if tuple(C.shape) != (M, N):
        raise ValueError("C must be %dx%d" % (M, N))
    with torch.cuda.device(C.device):
        rc = fn(*pre, transA.encode(), transB.encode(), M, N, K, float(alpha),
                ctypes.c_void_p(A.data_ptr()), _ld(A), ctypes.c_void_p(B.data_ptr()), _ld(B),
                float(beta), ctypes.c_void_p(C.data_ptr()), _ld(C), _stream(stream, C.device))
    _lib.check(rc, where)
    return C


def sgemm(A, B, C=None, transA: str = "N", transB: str = "N", alpha: float = 1.0, beta: float = 0.0,
          variant: int | None = None, stream=None):
    """C <- alpha * op(A) @ op(B) + beta * C on CUDA float32 row-major tensors.

    ``variant=None`` goes through the runtime selector (pt_sgemm); an int runs
    that registry variant (pt_sgemm_variant).  C is allocated when omitted
    (then beta must be 0).
    """
    import torch
    M, N, _ = _dims(A, B, transA, transB)
    if C is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs C")
        C = torch.empty((M, N), device=A.device, dtype=torch.float32)
    if variant is None:
        return _call(_l().pt_sgemm, "pt_sgemm", A, B, C, transA, transB, alpha, beta, stream)
    return _call(_l().pt_sgemm_variant, "pt_sgemm_variant", A, B, C, transA, transB, alpha, beta, stream,
                 pre=(int(variant),))


def reference(A, B, C=None, transA: str = "N", transB: str = "N", alpha: float = 1.0, beta: float = 0.0,
              stream=None):
    """The library's screening reference kernel (compensated dot product)."""
    import torch
    M, N, _ = _dims(A, B, transA, transB)
    if C is None:
        C = torch.empty((M, N), device=A.device, dtype=torch.float32)
    return _call(_l().pt_sgemm_reference, "pt_sgemm_reference", A, B, C, transA, transB, alpha, beta, stream)


def selected_variant(M: int, N: int, K: int, transA: str = "N", transB: str = "N", A=None, B=None, C=None) -> int:
    """Variant id pt_sgemm would launch (alignment from the tensors if given)."""
    def ptr_ld(t, cols):
        if t is None:
            return None, cols
        return ctypes.c_void_p(t.data_ptr()), _ld(t)
    pa, lda = ptr_ld(A, K if transA == "N" else M)
    pb, ldb = ptr_ld(B, N if transB == "N" else K)
    pc, ldc = ptr_ld(C, N)
    return _lib.check(_l().pt_selected_variant(transA.encode(), transB.encode(), M, N, K, pa, lda, pb, ldb,
                                               pc, ldc), "pt_selected_variant")


def device_status() -> int:
    return _l().pt_device_status()


def shutdown() -> None:
    """Frees the library's device workspaces and unloads the manifest."""
    _lib.check(_l().pt_shutdown(), "pt_shutdown")


def debug_streamk_wait(limit_ns: int = 0, never_ready: bool = False) -> None:
    """Failure-path hook of the stream-K hand-over wait (see the header)."""
    _lib.check(_l().pt_debug_streamk_wait(int(limit_ns), int(bool(never_ready))), "pt_debug_streamk_wait")


def streamk_segments(tiles: int, nchunks: int, units: int, unit: int) -> list:
    """The (tile, first chunk, end chunk) segments stream-K unit `unit` of
    `units` processes, in its visiting order (the kernels' own partition)."""
    n = _l().pt_debug_streamk_segments(tiles, nchunks, units, unit, None, 0)
    _lib.check(min(n, 0), "pt_debug_streamk_segments")
    buf = (ctypes.c_int * max(3, 3 * n))()
    _lib.check(min(_l().pt_debug_streamk_segments(tiles, nchunks, units, unit, buf, n), 0),
               "pt_debug_streamk_segments")
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]


def kernel_timer_start() -> None:
    """Starts timing the main GEMM kernel of every sgemm call on this thread."""
    _lib.check(_l().pt_kernel_timer_start(), "pt_kernel_timer_start")


def kernel_timer_stop():
    """Waits for the timed launches; returns (total milliseconds, launches)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    _lib.check(_l().pt_kernel_timer_stop(ctypes.byref(ms), ctypes.byref(n)), "pt_kernel_timer_stop")
    return ms.value, n.value


# ---- portability tuning --------------------------------------------------------------
def _shapes(shapes):
    arr = (Shape * len(shapes))()
    for i, s in enumerate(shapes):
        m, n, k = s[:3]
        ta = s[3] if len(s) > 3 else "N"
        tb = s[4] if len(s) > 4 else "N"
        arr[i] = Shape(m, n, k, ta.encode(), tb.encode())
    return arr


def tune(shapes, table_path: str, ids=None, warmup: int = 2, reps_min: int = 5, reps_max: int = 50,
         target_ms: float = 5.0, seed: int = 1, resume: bool = False, tol: float = 2e-6,
         pool_bytes: int = 1 << 30, verbose: bool = False, fail_launch: int = 0) -> None:
    """Timing table for ``shapes`` ((M, N, K[, transA, transB]) tuples) x variants.
    ``fail_launch`` (testing): the n-th variant launch reports a failure."""
    opts = TuneOpts(warmup, reps_min, reps_max, target_ms, seed, int(resume), tol, pool_bytes, int(verbose),
                    int(fail_launch))
    arr = _shapes(shapes)
    if ids is None:
        idp, nid = None, 0
    else:
        idp = (ctypes.c_int * len(ids))(*ids)
        nid = len(ids)
    _lib.check(_l().pt_tune(arr, len(shapes), idp, nid, ctypes.byref(opts), table_path.encode()), "pt_tune")


def select(table_path: str, train=None, k: int = 1, method: int = PT_SELECT_AUTO, seed: int = 0,
           manifest: str | None = None):
    """PortabilityTune over the table's training shapes: (ids, training geomean)."""
    train = list(train or [])
    tr = (ctypes.c_int * max(1, len(train)))(*train)
    out = (ctypes.c_int * k)()
    g = ctypes.c_double()
    _lib.check(_l().pt_select(table_path.encode(), tr, len(train), k, method, seed, out, ctypes.byref(g),
                              manifest.encode() if manifest else None), "pt_select")
    return [i for i in out if i >= 0], g.value


def score(table_path: str, shapes, ids=None, mode: int = PT_SCORE_BEST_OF_SET, manifest: str | None = None) -> float:
    """Geomean of t_best / t(chosen) over the given table shape indices."""
    shapes = list(shapes)
    sp = (ctypes.c_int * max(1, len(shapes)))(*shapes)
    ids = list(ids or [])
    ip = (ctypes.c_int * max(1, len(ids)))(*ids)
    g = ctypes.c_double()
    _lib.check(_l().pt_score(table_path.encode(), ip, len(ids), sp, len(shapes), mode,
                             manifest.encode() if manifest else None, ctypes.byref(g)), "pt_score")
    return g.value


def table_shapes(table_path: str) -> list:
    n = ctypes.c_int()
    _lib.check(_l().pt_table_shapes(table_path.encode(), ctypes.byref(n)), "pt_table_shapes")
    out = []
    for i in range(n.value):
        s = Shape()
        _lib.check(_l().pt_table_shape(table_path.encode(), i, ctypes.byref(s)), "pt_table_shape")
        out.append((s.m, s.n, s.k, s.transA.decode(), s.transB.decode()))
    return out


def grouped_problems(items, plan: bool = True):
    """Descriptor array for pt_sgemm_grouped from (A, B, C, transA, transB,
    alpha, beta) tuples of CUDA tensors; tiles from the runtime selector."""
    arr = (_lib.Problem * len(items))()
    for i, (A, B, C, ta, tb, alpha, beta) in enumerate(items):
        M, N, K = _dims(A, B, ta, tb)
        arr[i] = _lib.Problem(M, N, K, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C),
                              float(alpha), float(beta), ta.encode(), tb.encode(), 0, 3)
    if plan:
        _lib.check(_l().pt_grouped_plan(arr, len(items)), "pt_grouped_plan")
    return arr


def upload_problems(arr, device=None):
    """Device copy of a descriptor array (a uint8 CUDA tensor)."""
    import torch
    dev = device or torch.device("cuda", torch.cuda.current_device())
    return torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(dev)


def sgemm_grouped(arr, ddesc=None, stream=None, device=None):
    """One persistent launch over a descriptor array (see grouped_problems).
    ``ddesc`` is its device copy (upload_problems); made here when omitted.
    Returns the device copy; keep it alive and unchanged until the launch has
    completed (for a captured CUDA graph: as long as the graph is replayed)."""
    import torch
    dev = device or torch.device("cuda", torch.cuda.current_device())
    if ddesc is None:
        ddesc = upload_problems(arr, dev)
    with torch.cuda.device(dev):
        _lib.check(_l().pt_sgemm_grouped(arr, ctypes.c_void_p(ddesc.data_ptr()), len(arr), _stream(stream, dev)),
                   "pt_sgemm_grouped")
    return ddesc


def load_manifest(path: str | None) -> None:
    _lib.check(_l().pt_load_manifest(path.encode() if path else None), "pt_load_manifest")
