"""Counter-based SplitMix64 input generator.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) advances a 64-bit state by the golden-ratio
increment 0x9E3779B97F4A7C15 and passes it through a fixed finaliser.  The
i-th output (i >= 0) of the sequence seeded with ``seed`` is therefore
``mix(seed + (i + 1) * gamma)``; computing it from (seed, i) directly makes the
generator counter-based, so any element of any matrix can be produced
independently and in parallel.

Every matrix used by the tests, the tuner workloads and the benchmark is drawn
from here on the host, in FP32, and the same bits are handed to the CPU oracle
and copied to the device.
"""

from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_PAR_MIN = 1 << 20


def _workers():
    return max(1, min(32, os.cpu_count() or 1))

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, index) -> np.ndarray:
    """Outputs number ``index`` (0-based, array-like) of SplitMix64(seed)."""
    idx = np.asarray(index, dtype=np.uint64)
    base = np.uint64(seed & _MASK64)
    with np.errstate(over="ignore"):
        z = base + (idx + np.uint64(1)) * GAMMA
        return _mix(z)


def _bits(seed: int, n: int, offset: int = 0) -> np.ndarray:
    return splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n FP32 values uniform on [-1, 1): 2*(x>>40)/2^24 - 1, exact in FP32."""
    x = _bits(seed, n, offset)
    u = (x >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
    return (2.0 * u - 1.0).astype(np.float32)


def small_ints(seed: int, n: int, offset: int = 0, lo: int = -8, hi: int = 8) -> np.ndarray:
    """n FP32 integers uniform on [lo, hi]."""
    x = _bits(seed, n, offset)
    span = np.uint64(hi - lo + 1)
    return ((x >> np.uint64(32)) % span).astype(np.int64).astype(np.float32) + np.float32(lo)


def normal(seed: int, n: int, offset: int = 0, std: float = 1.0) -> np.ndarray:
    """n FP32 normals N(0, std^2): Box-Muller in FP64 on outputs 2i, 2i+1."""
    x = _bits(seed, 2 * n, 2 * offset)
    u1 = ((x[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (x[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return (z * std).astype(np.float32)


def log_uniform_signed(seed: int, n: int, offset: int = 0, lo_exp: float = -10.0,
                       hi_exp: float = 10.0) -> np.ndarray:
    """n FP32 values s * 2^e, s a random sign, e uniform on [lo_exp, hi_exp)."""
    x = _bits(seed, n, offset)
    sign = np.where((x & np.uint64(1)) == 1, -1.0, 1.0)
    u = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    e = lo_exp + (hi_exp - lo_exp) * u
    return (sign * np.exp2(e)).astype(np.float32)


_KINDS = {
    "uniform": uniform_pm1,
    "ints": small_ints,
    "normal": normal,
    "logu": log_uniform_signed,
}


def matrix(kind: str, seed: int, rows: int, cols: int, ld: int | None = None, **kw) -> np.ndarray:
    """A rows x cols row-major FP32 matrix (leading dimension ``ld`` >= cols).

    Padding columns (ld > cols) are filled with NaN so that a kernel which
    reads outside the logical matrix poisons its result.
    """
    ld = cols if ld is None else ld
    if ld < cols:
        raise ValueError("ld < cols")
    n = rows * cols
    fn = _KINDS[kind]
    if n >= _PAR_MIN:
        # Element i depends only on (seed, i): chunks are generated in parallel
        # threads (numpy releases the GIL) and give the same values.
        chunk = -(-n // _workers())
        starts = list(range(0, n, chunk))
        with ThreadPoolExecutor(max_workers=len(starts)) as ex:
            parts = list(ex.map(lambda s0: fn(seed, min(chunk, n - s0), offset=s0, **kw), starts))
        vals = np.concatenate(parts).reshape(rows, cols)
    elif n:
        vals = fn(seed, n, **kw).reshape(rows, cols)
    else:
        vals = np.zeros((rows, cols), np.float32)
    if ld == cols:
        return np.ascontiguousarray(vals)
    out = np.full((rows, ld), np.nan, dtype=np.float32)
    out[:, :cols] = vals
    return out
