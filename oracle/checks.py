"""Normalised error used by every parity test (test infrastructure only).

e = max |C - C_ref| / (K * max|A| * max|B| * |alpha| + |beta| * max|C_in|)

The denominator bounds |C_ref| for any inputs with those maxima, so e is the
error relative to the largest result the inputs allow.  At alpha = 1 and
beta = 0 it is max|C - C_ref| / (K * max|A| * max|B|).  Bounds: 2e-6 for FP32
SIMT and 3xTF32, 2e-3 for plain TF32.
"""

from __future__ import annotations

import numpy as np

TOL_FP32 = 2e-6
TOL_3XTF32 = 2e-6
TOL_TF32 = 2e-3


def normalised_error(C, C_ref, K, maxA, maxB, alpha=1.0, beta=0.0, maxC=0.0) -> float:
    C = np.asarray(C, dtype=np.float64)
    C_ref = np.asarray(C_ref, dtype=np.float64)
    if C.shape != C_ref.shape:
        raise ValueError("shape mismatch %s vs %s" % (C.shape, C_ref.shape))
    if C.size == 0:
        return 0.0
    if not np.all(np.isfinite(C)):
        return float("inf")
    denom = K * float(maxA) * float(maxB) * abs(float(alpha)) + abs(float(beta)) * float(maxC)
    diff = float(np.max(np.abs(C - C_ref)))
    if denom == 0.0:
        return 0.0 if diff == 0.0 else float("inf")
    return diff / denom
