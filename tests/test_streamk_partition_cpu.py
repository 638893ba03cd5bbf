"""CPU: the stream-K work partition of the tensor-core versions, taken from
the kernels' own partition code through pt_debug_streamk_segments (no device
work).  A unit is a CTA, or a CTA pair in the pair versions.

For every configuration the segments of all units must cover each (tile,
k-chunk) exactly once; whole tiles come first, in the strided order of a
persistent grid; a tile that several units share is finished by the unit
that owns its last chunk, every other unit that contributes to it has a
lower index (a finisher only ever waits for units dispatched before it), and
the finishing segment that waits for partial tiles is the last segment its
unit visits (so nothing of the unit's own work queues behind that wait).
"""

import itertools

import pytest

pt = pytest.importorskip("paper_2507_15277_gb300")

CONFIGS = [(tiles, nch, units)
           for tiles, nch, units in itertools.product((1, 2, 5, 64, 100, 128, 152, 256, 511, 512, 1024),
                                                      (1, 2, 3, 4, 16, 17, 64),
                                                      (1, 2, 38, 64, 76, 151, 152))
           if tiles * nch <= 70000]


def _partition(tiles, nch, units):
    return [pt.streamk_segments(tiles, nch, units, u) for u in range(units)]


@pytest.mark.parametrize("tiles,nch,units", CONFIGS)
def test_streamk_partition_covers_once_and_waits_only_on_earlier_units(tiles, nch, units):
    segs = _partition(tiles, nch, units)
    owner = {}
    for u, ss in enumerate(segs):
        for (t, c0, c1) in ss:
            assert 0 <= t < tiles and 0 <= c0 < c1 <= nch, (u, t, c0, c1)
            for c in range(c0, c1):
                assert (t, c) not in owner, ("chunk twice", t, c)
                owner[(t, c)] = u
    assert len(owner) == tiles * nch
    full_waves = tiles // units
    ndp = full_waves - 1 if full_waves >= 2 else 0
    for u, ss in enumerate(segs):
        # whole tiles first: u, u + units, ... for all but the last full wave
        assert ss[:ndp] == [(u + i * units, 0, nch) for i in range(ndp)]
        for i, (t, c0, c1) in enumerate(ss):
            if c0 > 0 and c1 == nch:
                # this unit finishes a shared tile: it waits for the units
                # holding chunks 0 .. c0 - 1, all of lower index, and this is
                # its last segment
                assert i == len(ss) - 1, (u, ss)
                assert all(owner[(t, c)] < u for c in range(c0)), (u, t)
            elif c1 < nch:
                # a contributor: the tile's finisher has a higher index
                assert owner[(t, nch - 1)] > u, (u, t)


def test_streamk_partition_balances_the_shared_part():
    # the shared chunks differ by at most one between units
    tiles, nch, units = 256, 16, 76   # the 256 x 256 pair tiles of a 4096^3 GEMM on 76 pairs
    ndp = tiles // units - 1
    shared = [sum(c1 - c0 for (t, c0, c1) in ss[ndp:]) for ss in _partition(tiles, nch, units)]
    assert max(shared) - min(shared) <= 1
    assert sum(shared) == (tiles - ndp * units) * nch


def test_streamk_segments_argument_errors():
    lib = pt._lib.lib()
    for args in ((0, 1, 1, 0), (1, 0, 1, 0), (1, 1, 0, 0), (1, 1, 2049, 0), (4, 4, 2, 2), (4, 4, 2, -1)):
        assert lib.pt_debug_streamk_segments(*args, None, 0) == pt._lib.PT_EINVAL
    assert lib.pt_debug_streamk_segments(4, 4, 2, 0, None, 1) == pt._lib.PT_EINVAL
    assert lib.pt_debug_streamk_segments(4, 4, 2, 0, None, 0) >= 1
