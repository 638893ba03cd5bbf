"""Split-precision planes of FP32 values -- TEST INFRASTRUCTURE ONLY.

The tensor-core versions of the SGEMM family (an extension: the paper's
kernels are FP32 only) write each FP32 operand as a sum of lower-precision
planes and drop the smallest cross products:

  3xTF32: x = hi + lo, hi = RN_tf32(x), lo = RN_tf32(x - hi);
          a*b ~ hi_a*hi_b + hi_a*lo_b + lo_a*hi_b   (lo_a*lo_b dropped)
  BF16x3: x = b0 + b1 + b2, b0 = RN_bf16(x), b1 = RN_bf16(x - b0),
          b2 = RN_bf16(x - b0 - b1);
          a*b ~ sum of a_i*b_j over i + j <= 2       (a1b2, a2b1, a2b2 dropped)

RN_p rounds to the nearest value with p significant bits, ties to even
(TF32: p = 11, BF16: p = 8; the FP32 exponent range is kept).  This module
states the rounding arithmetically (frexp / ldexp and numpy's round-half-even)
so that tests can show which planes and which products a set of inputs
exercises.  Only the tests use it; the library splits with bit operations of
its own.
"""

from __future__ import annotations

import numpy as np

P_TF32 = 11
P_BF16 = 8


def round_sig(x, p: int) -> np.ndarray:
    """x (FP32 values) rounded to p significant bits, ties to even, in FP64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                     # x = m * 2^e, 0.5 <= |m| < 1
    r = np.round(np.ldexp(m, p))           # p-bit integer significand, half to even
    return np.ldexp(r, e - p)


def tf32x2_planes(x):
    """(hi, lo) of the 3xTF32 split, FP64 arrays holding TF32 values."""
    x = np.asarray(x, dtype=np.float64)
    hi = round_sig(x, P_TF32)
    lo = round_sig(x - hi, P_TF32)
    return hi, lo


def bf16x3_planes(x):
    """(b0, b1, b2) of the BF16x3 split, FP64 arrays holding BF16 values."""
    x = np.asarray(x, dtype=np.float64)
    b0 = round_sig(x, P_BF16)
    b1 = round_sig(x - b0, P_BF16)
    b2 = round_sig(x - b0 - b1, P_BF16)
    return b0, b1, b2


BF16X3_KEPT = [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 0)]
BF16X3_DROPPED = [(1, 2), (2, 1), (2, 2)]
TF32X3_KEPT = [(0, 0), (0, 1), (1, 0)]
TF32X3_DROPPED = [(1, 1)]
