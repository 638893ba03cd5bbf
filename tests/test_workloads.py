"""The seeded input generators (shared by the oracle side and the GPU side)."""

import numpy as np

from workloads import (grouped_problems, matrix, parity_split, random_split,
                       splitmix64, sweep_shapes, uniform_pm1)


def test_splitmix64_published_vectors():
    # First outputs of SplitMix64 seeded with 1234567 (reference implementation
    # by Vigna, the generator of Steele, Lea and Flood, OOPSLA 2014).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(x) for x in splitmix64(1234567, np.arange(5))] == want


def test_counter_based_access():
    a = splitmix64(7, np.arange(100))
    b = splitmix64(7, np.array([5, 99, 0]))
    assert list(b) == [a[5], a[99], a[0]]


def test_uniform_values_exact_on_grid():
    x = uniform_pm1(1, 100000)
    assert x.dtype == np.float32
    assert x.min() >= -1.0 and x.max() < 1.0
    y = (x.astype(np.float64) + 1.0) * 2.0 ** 23
    assert np.all(y == np.round(y))
    assert abs(float(x.mean())) < 0.01


def test_ints_and_padding():
    a = matrix("ints", 3, 10, 6, ld=9)
    assert np.all(np.isnan(a[:, 6:]))
    v = a[:, :6]
    assert v.min() >= -8 and v.max() <= 8 and np.all(v == np.round(v))


def test_sweep_and_split():
    shapes = sweep_shapes()
    assert len(shapes) == 64 and len(set(shapes)) == 64
    tr, he = parity_split()
    assert len(tr) == 32 and len(he) == 32 and not set(tr) & set(he)
    for dim in range(3):
        for size in (128, 512, 1024, 4096):
            assert sum(shapes[i][dim] == size for i in tr) == 8
    tr2, he2 = random_split(0)
    assert len(tr2) == 32 and sorted(tr2 + he2) == list(range(64))
    assert random_split(0) == (tr2, he2) and random_split(1) != (tr2, he2)


def test_grouped_problem_sizes():
    probs = grouped_problems()
    assert len(probs) == 512
    d = np.array(probs)
    assert d.min() >= 32 and d.max() <= 2048 and np.all(d % 8 == 0)
