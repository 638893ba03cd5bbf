"""Persistent grouped SGEMM (many uneven problems in one launch): SIMT tiles
in the grouped kernel, and problems given the tensor-core tile in the grouped
3xF16 kernel (split into tiled planes, one persistent tensor-core launch)."""

import ctypes

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import grouped_problems, matrix

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")
from paper_2507_15277_gb300 import _lib  # noqa: E402


def _store(X, t):
    return np.ascontiguousarray(X.T if t == "T" else X)


def test_grouped_argument_validation_on_host():
    lib = _lib.lib()
    arr = (_lib.Problem * 2)()
    arr[0] = _lib.Problem(8, 8, 8, 16, 8, 16, 8, 16, 8, 1.0, 0.0, b"N", b"N", 0, 0)
    arr[1] = _lib.Problem(8, 8, 8, 16, 8, 16, 8, 16, 8, 1.0, 0.0, b"N", b"X", 0, 0)
    assert lib.pt_sgemm_grouped(arr, ctypes.c_void_p(16), 2, None) == _lib.PT_EINVAL
    arr[1] = _lib.Problem(8, 8, 8, 16, 7, 16, 8, 16, 8, 1.0, 0.0, b"N", b"N", 0, 0)   # lda < K
    assert lib.pt_sgemm_grouped(arr, ctypes.c_void_p(16), 2, None) == _lib.PT_EINVAL
    arr[1] = _lib.Problem(8, 8, 8, 20, 8, 16, 8, 16, 8, 1.0, 0.0, b"N", b"N", 0, 2)   # tile 2 needs alignment
    assert lib.pt_sgemm_grouped(arr, ctypes.c_void_p(16), 2, None) == _lib.PT_EINVAL
    arr[1] = _lib.Problem(8, 8, 8, 16, 8, 16, 8, 16, 8, 1.0, 0.0, b"N", b"N", 0, 9)   # unknown tile
    assert lib.pt_sgemm_grouped(arr, ctypes.c_void_p(16), 2, None) == _lib.PT_EINVAL
    arr[1] = _lib.Problem(8, 8, 0, 16, 8, 16, 8, 16, 8, 1.0, 0.0, b"N", b"N", 0, 4)   # tensor-core tile, K = 0
    assert lib.pt_sgemm_grouped(arr, ctypes.c_void_p(16), 2, None) == _lib.PT_EINVAL
    assert lib.pt_sgemm_grouped(arr, None, 5000, None) == _lib.PT_EINVAL  # more than PT_GROUPED_MAX
    assert lib.pt_sgemm_grouped(arr, None, 0, None) == 0


@pytest.mark.gpu
def test_grouped_mixed_problems_bit_exact():
    dev = "cuda:0"
    rng = np.random.default_rng(1)
    specs = []
    for i in range(40):
        M, N, K = (int(x) for x in rng.integers(1, 300, size=3))
        ta, tb = rng.choice(["N", "T"]), rng.choice(["N", "T"])
        specs.append((M, N, K, ta, tb))
    specs += [(0, 5, 5, "N", "N"), (7, 9, 0, "N", "N"), (130, 70, 1, "T", "N")]
    items, refs, keep = [], [], []
    for i, (M, N, K, ta, tb) in enumerate(specs):
        A = matrix("ints", 100 + i, M, K)
        B = matrix("ints", 200 + i, K, N)
        C0 = matrix("ints", 300 + i, M, N)
        alpha, beta = (1.0, 0.0) if i % 3 else (2.0, -1.0)
        As, Bs = _store(A, ta), _store(B, tb)
        Ad = torch.from_numpy(As).to(dev)
        Bd = torch.from_numpy(Bs).to(dev)
        Cd = torch.from_numpy(C0).to(dev)
        if i % 5 == 4 and M > 1 and K > 1:  # an odd leading dimension: generic tile
            Ad = torch.from_numpy(np.ascontiguousarray(np.pad(As, ((0, 0), (0, 1))))).to(dev)[:, :As.shape[1]]
        items.append((Ad, Bd, Cd, ta, tb, alpha, beta))
        refs.append(og.gemm(As, Bs, ta, tb, alpha=alpha, beta=beta, C=C0) if M and N else np.zeros((M, N)))
        keep.append((Ad, Bd))
    arr = pt.grouped_problems(items)
    tiles = {arr[i].tile for i in range(len(items))}
    assert 3 in tiles
    d = pt.sgemm_grouped(arr)
    torch.cuda.synchronize()
    for (Ad, Bd, Cd, *_), ref in zip(items, refs):
        assert np.array_equal(Cd.cpu().numpy().astype(np.float64), ref)
    del d


@pytest.mark.gpu
def test_grouped_512_problems_sampled_and_graph_replay():
    dev = "cuda:0"
    probs = grouped_problems()
    items, hostAB = [], []
    for i, (M, N, K) in enumerate(probs):
        A = matrix("uniform", 5000 + i, M, K)
        B = matrix("uniform", 6000 + i, K, N)
        hostAB.append((A, B))
        items.append((torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev),
                      torch.empty((M, N), device=dev), "N", "N", 1.0, 0.0))
    arr = pt.grouped_problems(items)
    d = pt.sgemm_grouped(arr)
    torch.cuda.synchronize()
    for i in list(range(0, 512, 37)) + [511]:
        A, B = hostAB[i]
        M, N, K = probs[i]
        rows = list(range(0, M, max(1, M // 16)))
        ref = og.gemm(A, B, rows=rows)
        got = items[i][2][rows].cpu().numpy()
        assert normalised_error(got, ref, K, np.abs(A).max(), np.abs(B).max()) <= TOL_FP32, i
    snap = [it[2].clone() for it in items[:8]]
    for it in items[:8]:
        it[2].zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pt.sgemm_grouped(arr, ddesc=d, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for it, ref in zip(items[:8], snap):
        assert torch.equal(it[2], ref)
    del d


def _tc_items(specs, kind, dev, seed0):
    items, refs, keep = [], [], []
    for i, (M, N, K, ta, tb) in enumerate(specs):
        if kind == "wide":
            from workloads import wide_int_operands
            A, B, _ = wide_int_operands(seed0 + i, M, N, K)
        else:
            A = matrix(kind, seed0 + i, M, K)
            B = matrix(kind, seed0 + 1000 + i, K, N)
        C0 = matrix("ints", seed0 + 2000 + i, M, N)
        alpha, beta = (1.0, 0.0) if i % 3 else (2.0, -1.0)
        As, Bs = _store(A, ta), _store(B, tb)
        Ad, Bd, Cd = (torch.from_numpy(x).to(dev) for x in (As, Bs, C0))
        items.append((Ad, Bd, Cd, ta, tb, alpha, beta))
        refs.append((og.gemm(As, Bs, ta, tb, alpha=alpha, beta=beta, C=C0), A, B, C0, alpha, beta, K))
    return items, refs


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["ints", "wide"])
def test_grouped_tensor_core_tile_bit_exact(kind):
    # Ragged M, N (several 128-row tiles and a tail), K spanning 1 to 5 chunks
    # with a ragged end, every transpose pair; every other problem stays on a
    # SIMT tile in the same call.  Exact-integer inputs: bit for bit.
    dev = "cuda:0"
    rng = np.random.default_rng(7)
    specs = []
    for i in range(24):
        M = int(rng.integers(1, 400)) if kind == "ints" else int(rng.integers(200, 400))
        N, K = int(rng.integers(1, 400)), int(rng.integers(1, 600))
        if kind == "wide":
            K = int(rng.integers(64, 1100))
        specs.append((M, N, K, ["N", "T"][i % 2], ["N", "T"][(i // 2) % 2]))
    items, refs = _tc_items(specs, kind, dev, 700)
    arr = pt.grouped_problems(items)
    for i in range(len(items)):
        if i % 4 != 3:
            arr[i].tile = 4
    d = pt.sgemm_grouped(arr)
    torch.cuda.synchronize()
    for i, ((Ad, Bd, Cd, *_), (ref, *_r)) in enumerate(zip(items, refs)):
        got = Cd.cpu().numpy().astype(np.float64)
        assert np.array_equal(got, ref), (i, specs[i], arr[i].tile, int(np.sum(got != ref)))
    assert pt.device_status() == 0
    del d


@pytest.mark.gpu
def test_grouped_512_problems_with_tensor_core_tiles_against_oracle():
    # The grouped workload (512 problems, M, N, K log-uniform in [32, 2048]):
    # problems of 2^27 multiply-adds or more on the tensor-core tile, the rest
    # on SIMT tiles; sampled rows against the oracle, then a graph replay.
    dev = "cuda:0"
    probs = grouped_problems()
    items, hostAB = [], []
    for i, (M, N, K) in enumerate(probs):
        A = matrix("uniform", 5000 + i, M, K)
        B = matrix("uniform", 6000 + i, K, N)
        hostAB.append((A, B))
        items.append((torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev),
                      torch.empty((M, N), device=dev), "N", "N", 1.0, 0.0))
    arr = pt.grouped_problems(items)
    big = [i for i, (M, N, K) in enumerate(probs) if M * N * K >= 1 << 27]
    for i in big:
        arr[i].tile = 4
    assert 20 < len(big) < 500
    d = pt.sgemm_grouped(arr)
    torch.cuda.synchronize()
    for i in sorted(set(big[::7] + list(range(0, 512, 41)))):
        A, B = hostAB[i]
        M, N, K = probs[i]
        rows = list(range(0, M, max(1, M // 16)))
        ref = og.gemm(A, B, rows=rows)
        got = items[i][2][rows].cpu().numpy()
        assert normalised_error(got, ref, K, np.abs(A).max(), np.abs(B).max()) <= TOL_FP32, (i, arr[i].tile)
    snap = [items[i][2].clone() for i in big[:6]]
    for i in big[:6]:
        items[i][2].fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pt.sgemm_grouped(arr, ddesc=d, stream=s)   # the stream's workspace grows outside the capture
        s.synchronize()
        for i in big[:6]:
            items[i][2].fill_(float("nan"))
        with torch.cuda.graph(g, stream=s):
            pt.sgemm_grouped(arr, ddesc=d, stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for i, ref in zip(big[:6], snap):
        assert torch.equal(items[i][2], ref)
    assert pt.device_status() == 0
    del d
