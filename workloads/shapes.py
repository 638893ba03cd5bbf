"""Shape lists of the synthetic workloads.

The portability sweep is the paper's regular input grid (Section V-B, Table 4):
every (M, N, K) whose three extents each come from one size set, giving 64
square and rectangular products.  The size set here is {128, 512, 1024, 4096}.
"""

from __future__ import annotations

import itertools

import numpy as np

from .rng import splitmix64

SWEEP_SIZES = (128, 512, 1024, 4096)


def sweep_shapes(sizes=SWEEP_SIZES):
    """All (M, N, K) over ``sizes``^3, M slowest, K fastest (index order)."""
    return [tuple(s) for s in itertools.product(sizes, sizes, sizes)]


def parity_split(sizes=SWEEP_SIZES):
    """Train/held-out split of the sweep: (i_m + i_n + i_k) even -> train.

    Balanced: every size appears equally often in each half, in every
    dimension.  Returns (train_indices, heldout_indices).
    """
    n = len(sizes)
    train, held = [], []
    for idx, (im, i_n, ik) in enumerate(itertools.product(range(n), range(n), range(n))):
        (train if (im + i_n + ik) % 2 == 0 else held).append(idx)
    return train, held


def random_split(seed: int, n_shapes: int = 64, n_train: int = 32):
    """A seeded random train/held-out split (Fisher-Yates driven by SplitMix64)."""
    perm = list(range(n_shapes))
    draws = splitmix64(seed, np.arange(n_shapes, dtype=np.uint64))
    for i in range(n_shapes - 1, 0, -1):
        j = int(draws[i] % np.uint64(i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return sorted(perm[:n_train]), sorted(perm[n_train:])


def split_precision_shapes():
    """Square 1024/4096/8192 and the two skinny 8192/256 products."""
    return [(1024, 1024, 1024), (4096, 4096, 4096), (8192, 8192, 8192),
            (8192, 8192, 256), (256, 8192, 8192)]


def grouped_problems(seed: int = 5, count: int = 512, lo: int = 32, hi: int = 2048):
    """``count`` problems with M, N, K = 8*round(2^U[5,11] / 8) clamped to [lo, hi]."""
    x = splitmix64(seed, np.arange(3 * count, dtype=np.uint64))
    u = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    v = np.exp2(5.0 + 6.0 * u)
    d = np.clip(8 * np.rint(v / 8.0), lo, hi).astype(np.int64)
    return [tuple(int(t) for t in d[3 * i:3 * i + 3]) for i in range(count)]
