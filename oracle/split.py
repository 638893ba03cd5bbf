"""Split-precision planes of FP32 values -- TEST INFRASTRUCTURE ONLY.

The tensor-core versions of the SGEMM family (an extension: the paper's
kernels are FP32 only) write each FP32 operand as a sum of lower-precision
planes and drop the smallest cross products:

  3xTF32: x = hi + lo, hi = RN_tf32(x), lo = RN_tf32(x - hi);
          a*b ~ hi_a*hi_b + hi_a*lo_b + lo_a*hi_b   (lo_a*lo_b dropped)
  BF16x3: x = b0 + b1 + b2, b0 = RN_bf16(x), b1 = RN_bf16(x - b0),
          b2 = RN_bf16(x - b0 - b1);
          a*b ~ sum of a_i*b_j over i + j <= 2       (a1b2, a2b1, a2b2 dropped)

  3xF16 (scaled): k is cut into chunks of 256 values; chunk c of row i of
          op(A) is multiplied by 2^S with S = 14 - floor(log2 m), m its
          largest magnitude, clamped to [-63, 63] (63 when m = 0); chunk c of
          a group of 32 consecutive columns of op(B) likewise, m over the
          group's chunk.  Then x' = h0 + h1 with h0 = RN_f16(x'),
          h1 = RN_f16(x' - h0) and the products kept as in 3xTF32; each
          chunk's sum is multiplied back by 2^-S_A 2^-S_B.

RN_p rounds to the nearest value with p significant bits, ties to even
(TF32: p = 11, BF16: p = 8; the FP32 exponent range is kept).  RN_f16 is
IEEE binary16 rounding (11 significant bits, subnormals below 2^-14),
taken from numpy's float16 conversion.  This module
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


def f16_chunk_scales(X, group: int = 1, chunk: int = 256) -> np.ndarray:
    """Exponents S[g, c] of the 3xF16 split of X (rows x K), for groups of
    `group` consecutive rows (1 for op(A); 32 for the rows of op(B)^T) and
    chunks of `chunk` values of k: 2^S brings the largest magnitude of the
    group's chunk into [2^14, 2^15)."""
    X = np.abs(np.asarray(X, dtype=np.float64))
    rows, K = X.shape
    ng, nch = -(-rows // group), -(-K // chunk)
    S = np.empty((ng, nch), dtype=np.int64)
    for g in range(ng):
        for c in range(nch):
            m = X[g * group:(g + 1) * group, c * chunk:(c + 1) * chunk].max(initial=0.0)
            S[g, c] = 63 if m == 0 else int(np.clip(14 - np.floor(np.log2(m)), -63, 63))
    return S


def f16x2_planes_scaled(X, group: int = 1, chunk: int = 256):
    """(h0, h1, E) of the scaled 3xF16 split of the rows of X: h0 + h1 is
    X[r, k] * 2^E[r, k] on the FP16 grid (FP64 arrays), E[r, k] the scale
    exponent of r's group and k's chunk."""
    X = np.asarray(X, dtype=np.float64)
    S = f16_chunk_scales(X, group, chunk)
    E = np.repeat(np.repeat(S, group, axis=0), chunk, axis=1)[:X.shape[0], :X.shape[1]]
    xs = X * np.ldexp(1.0, E)
    with np.errstate(over="ignore", invalid="ignore"):   # beyond FP16's range: inf, as the kernel
        h0 = xs.astype(np.float16).astype(np.float64)
        h1 = (xs - h0).astype(np.float16).astype(np.float64)
    return h0, h1, E


BF16X3_KEPT = [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 0)]
BF16X3_DROPPED = [(1, 2), (2, 1), (2, 2)]
TF32X3_KEPT = [(0, 0), (0, 1), (1, 0)]
TF32X3_DROPPED = [(1, 1)]
