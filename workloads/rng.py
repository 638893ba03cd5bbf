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


def rank1_operands(M: int, N: int, K: int):
    """A (M x K) of ones and B (K x N) with B[k][j] = k: every entry of A*B is
    sum_{k<K} k = K(K-1)/2, a closed form (exact in FP32 for K <= 4096)."""
    A = np.ones((M, K), np.float32)
    B = np.repeat(np.arange(K, dtype=np.float32)[:, None], N, axis=1)
    return A, np.ascontiguousarray(B)


def _signed_ints(seed: int, n: int, lo: int, hi: int, odd: bool = False) -> np.ndarray:
    """n FP64 integers of magnitude uniform on [lo, hi) (odd ones only when
    ``odd``) with a random sign."""
    x = _bits(seed, n)
    if odd:
        mag = ((x >> np.uint64(33)) % np.uint64((hi - lo) // 2)) * np.uint64(2) + np.uint64(lo + 1)
    else:
        mag = (x >> np.uint64(33)) % np.uint64(hi - lo) + np.uint64(lo)
    sign = np.where((x & np.uint64(1)) == 1, -1.0, 1.0)
    return sign * mag.astype(np.float64)


def wide_int_operands(seed: int, M: int, N: int, K: int):
    """Integer operands with 18-, 9- and 1-bit entries whose exact product
    stays below 2^24 in every partial sum.

    Each k has a type t = k mod 3:
      t = 0: A[i][k] has magnitude in [2^17, 2^18) (18 bits), B[k][j] is +-1;
      t = 1: A[i][k] is +-1, B[k][j] has magnitude in [2^17, 2^18);
      t = 2: both are odd with magnitude in [2^8, 2^9) (9 bits).
    B is dense.  A[i][k] is non-zero only where (k - i) mod P is 0, 1 or 2,
    with P = max(64, ceil(K / 16)): row i meets at most 16 windows of three
    consecutive k (one of each type), so sum_k |A[i][k] B[k][j]| is below
    16 * 3 * 2^18 < 2^24, and every row offset of A touches a different k,
    so with M >= P every k of every operand is used.
    Returns (A, B, P).
    """
    P = max(64, -(-K // 16))
    t = np.arange(K) % 3
    big = _signed_ints(seed, M * K, 1 << 17, 1 << 18).reshape(M, K)
    mid = _signed_ints(seed + 1, M * K, 1 << 8, 1 << 9, odd=True).reshape(M, K)
    one = _signed_ints(seed + 2, M * K, 1, 2).reshape(M, K)
    A = np.where(t == 0, big, np.where(t == 1, one, mid))
    window = (np.arange(K)[None, :] - np.arange(M)[:, None]) % P < 3
    A = np.where(window, A, 0.0)
    bbig = _signed_ints(seed + 3, K * N, 1 << 17, 1 << 18).reshape(K, N)
    bmid = _signed_ints(seed + 4, K * N, 1 << 8, 1 << 9, odd=True).reshape(K, N)
    bone = _signed_ints(seed + 5, K * N, 1, 2).reshape(K, N)
    tk = t[:, None]
    B = np.where(tk == 0, bone, np.where(tk == 1, bbig, bmid))
    return np.ascontiguousarray(A.astype(np.float32)), np.ascontiguousarray(B.astype(np.float32)), P
