"""ctypes binding of libptsgemm.so (argument marshalling only).

Loading fails loudly when the library has not been built: there is no
fallback implementation of any entry point.
"""

from __future__ import annotations

import ctypes
import os

from .build import LIB

PT_OK = 0
PT_EINVAL = -1
PT_EUNSUPPORTED = -2
PT_ECUDA = -3
PT_EIO = -4
PT_EFORMAT = -5
PT_ETIMEOUT = -6

PT_LOADER_CPASYNC = 0
PT_LOADER_TMA = 1
PT_SCHED_TILE = 0
PT_SCHED_PERSISTENT = 1
PT_SCHED_STREAMK = 2

PT_SELECT_EXACT = 0
PT_SELECT_GREEDY_SWAP = 1
PT_SELECT_AUTO = 2
PT_SELECT_KMEANS = 3
PT_SELECT_TREE = 4

PT_SCORE_BEST_OF_SET = 0
PT_SCORE_SELECTOR = 1

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


class VariantDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "id", "bm", "bn", "bk", "wm", "wn", "tm", "tn", "kl", "vec", "stages", "splitk", "loader",
        "a_kmajor", "threads", "smem_bytes", "trans_mask", "kind", "fma2", "schedule")] + \
        [("name", ctypes.c_char * 96)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_ if n != "name"}
        d["name"] = self.name.decode()
        return d


class Shape(ctypes.Structure):
    _fields_ = [("m", _i64), ("n", _i64), ("k", _i64), ("transA", ctypes.c_char), ("transB", ctypes.c_char)]


class TuneOpts(ctypes.Structure):
    _fields_ = [("warmup", ctypes.c_int), ("reps_min", ctypes.c_int), ("reps_max", ctypes.c_int),
                ("target_ms", ctypes.c_double), ("seed", ctypes.c_uint64), ("resume", ctypes.c_int),
                ("tol", ctypes.c_double), ("pool_bytes", _i64), ("verbose", ctypes.c_int),
                ("fail_launch", _i64)]


class Problem(ctypes.Structure):
    _fields_ = [("m", _i64), ("n", _i64), ("k", _i64), ("A", _p), ("lda", _i64), ("B", _p), ("ldb", _i64),
                ("C", _p), ("ldc", _i64), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("transA", ctypes.c_char), ("transB", ctypes.c_char), ("reserved", ctypes.c_int16),
                ("tile", ctypes.c_int32)]


_GEMM_ARGS = [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, ctypes.c_float, _p, _i64, _p, _i64,
              ctypes.c_float, _p, _i64, _p]

# name -> (restype, argtypes); every export declared in include/pt_sgemm.h.
SIGNATURES = {
    "pt_last_error": (ctypes.c_char_p, []),
    "pt_last_error_arg": (ctypes.c_int, []),
    "pt_sgemm": (ctypes.c_int, _GEMM_ARGS),
    "pt_sgemm_variant": (ctypes.c_int, [ctypes.c_int] + _GEMM_ARGS),
    "pt_sgemm_reference": (ctypes.c_int, _GEMM_ARGS),
    "pt_num_variants": (ctypes.c_int, []),
    "pt_variant_desc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(VariantDesc)]),
    "pt_variant_by_name": (ctypes.c_int, [ctypes.c_char_p]),
    "pt_default_variant": (ctypes.c_int, []),
    "pt_tune_default_opts": (None, [ctypes.POINTER(TuneOpts)]),
    "pt_tune": (ctypes.c_int, [ctypes.POINTER(Shape), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                               ctypes.POINTER(TuneOpts), ctypes.c_char_p]),
    "pt_select": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double), ctypes.c_char_p]),
    "pt_score": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_char_p,
                                ctypes.POINTER(ctypes.c_double)]),
    "pt_table_shapes": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
    "pt_table_shape": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(Shape)]),
    "pt_load_manifest": (ctypes.c_int, [ctypes.c_char_p]),
    "pt_selected_variant": (ctypes.c_int, [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _p, _i64, _p, _i64,
                                           _p, _i64]),
    "pt_device_status": (ctypes.c_int, []),
    "pt_shutdown": (ctypes.c_int, []),
    "pt_kernel_timer_start": (ctypes.c_int, []),
    "pt_kernel_timer_stop": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "pt_sgemm_3xtf32_noalloc": (ctypes.c_int, _GEMM_ARGS),
    "pt_debug_streamk_wait": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int]),
    "pt_debug_streamk_segments": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "pt_grouped_plan": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int]),
    "pt_sgemm_grouped": (ctypes.c_int, [ctypes.POINTER(Problem), _p, ctypes.c_int, _p]),
}

_lib = None


def lib():
    """The loaded library; raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError("libptsgemm.so is not built (%s); run __graft_entry__.build() or "
                              "python -m paper_2507_15277_gb300.build" % LIB)
        handle = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


class PtError(RuntimeError):
    def __init__(self, code, where):
        l = lib()
        msg = (l.pt_last_error() or b"").decode(errors="replace")
        self.code = code
        self.arg = l.pt_last_error_arg()
        super().__init__("%s failed (%d): %s" % (where, code, msg))


def check(code, where):
    if code < 0:
        raise PtError(code, where)
    return code
