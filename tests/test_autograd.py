"""Y = X @ W as a torch.autograd.Function on the tuned SGEMM.

CPU part: the oracle's gradient formulas (dX = G W^T, dW = X^T G) against FP64
finite differences of the oracle loss sum(Y * G).  GPU part: the library's
forward/backward against the oracle, at 64x48x32 and at the full
X[4096,1024] @ W[1024,4096] size (sampled rows), with NT/TN shapes tuned and
selected through a manifest.
"""

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix


def _loss(X, W, G):
    return float(np.sum(og.gemm(X, W) * G.astype(np.float64)))


def _fd_grad_x(X, W, G, entries):
    """Central differences of the FP64 oracle loss; the perturbation is the
    exact FP32 difference of the perturbed inputs."""
    out = []
    for (i, k) in entries:
        h = np.float32(2.0 ** -8)
        Xp, Xm = X.copy(), X.copy()
        Xp[i, k] = X[i, k] + h
        Xm[i, k] = X[i, k] - h
        d = float(Xp[i, k]) - float(Xm[i, k])
        out.append((_loss(Xp, W, G) - _loss(Xm, W, G)) / d)
    return np.array(out)


def _fd_grad_w(X, W, G, entries):
    out = []
    for (k, j) in entries:
        h = np.float32(2.0 ** -8)
        Wp, Wm = W.copy(), W.copy()
        Wp[k, j] = W[k, j] + h
        Wm[k, j] = W[k, j] - h
        d = float(Wp[k, j]) - float(Wm[k, j])
        out.append((_loss(X, Wp, G) - _loss(X, Wm, G)) / d)
    return np.array(out)


SMALL = (64, 48, 32)  # M (rows of X), N (cols of W), K (inner)


def _small_inputs():
    M, N, K = SMALL
    X = matrix("normal", 41, M, K, std=0.02)
    W = matrix("normal", 42, K, N, std=0.02)
    G = matrix("normal", 43, M, N)
    return X, W, G


def test_oracle_gradients_match_finite_differences():
    X, W, G = _small_inputs()
    M, N, K = SMALL
    dX = og.gemm(G, W, "N", "T")      # G (MxN) @ W^T (NxK)
    dW = og.gemm(X, G, "T", "N")      # X^T (KxM) @ G (MxN)
    ex = [(i, k) for i in range(M) for k in range(K)]
    ew = [(k, j) for k in range(K) for j in range(N)]
    fx = _fd_grad_x(X, W, G, ex).reshape(M, K)
    fw = _fd_grad_w(X, W, G, ew).reshape(K, N)
    # The loss is linear in X and W: central differences are exact up to FP64
    # rounding of the loss (|loss terms| <= M*N*max|G*Y|).
    assert np.max(np.abs(fx - dX)) <= 1e-9
    assert np.max(np.abs(fw - dW)) <= 1e-9


@pytest.mark.gpu
def test_autograd_small_against_oracle_and_fd():
    torch = pytest.importorskip("torch")
    pt = pytest.importorskip("paper_2507_15277_gb300")
    from paper_2507_15277_gb300.autograd import matmul
    X, W, G = _small_inputs()
    M, N, K = SMALL
    Xd = torch.from_numpy(X).cuda().requires_grad_(True)
    Wd = torch.from_numpy(W).cuda().requires_grad_(True)
    Y = matmul(Xd, Wd)
    loss = (Y * torch.from_numpy(G).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    Yr = og.gemm(X, W)
    assert normalised_error(Y.detach().cpu().numpy(), Yr, K, np.abs(X).max(), np.abs(W).max()) <= TOL_FP32
    dX = og.gemm(G, W, "N", "T")
    dW = og.gemm(X, G, "T", "N")
    gX = Xd.grad.cpu().numpy()
    gW = Wd.grad.cpu().numpy()
    assert normalised_error(gX, dX, N, np.abs(G).max(), np.abs(W).max()) <= TOL_FP32
    assert normalised_error(gW, dW, M, np.abs(X).max(), np.abs(G).max()) <= TOL_FP32
    fx = _fd_grad_x(X, W, G, [(0, 0), (17, 5), (63, 31)])
    assert np.allclose(gX[[0, 17, 63], [0, 5, 31]], fx, rtol=0, atol=TOL_FP32 * N * np.abs(G).max() * np.abs(W).max())


@pytest.mark.gpu
def test_autograd_full_size_through_selector(tmp_path):
    torch = pytest.importorskip("torch")
    pt = pytest.importorskip("paper_2507_15277_gb300")
    from paper_2507_15277_gb300.autograd import matmul
    M, K, N = 4096, 1024, 4096
    shapes = [(M, N, K, "N", "N"), (M, K, N, "N", "T"), (K, N, M, "T", "N")]
    table = str(tmp_path / "t.csv")
    ids = list(range(0, pt.num_variants(), 6))
    pt.tune(shapes, table, ids=ids, reps_min=3, reps_max=5, target_ms=1.0)
    man = str(tmp_path / "m.json")
    kappa, _ = pt.select(table, [0, 1, 2], 3, manifest=man)
    pt.load_manifest(man)
    try:
        for (m, n, k, ta, tb) in shapes:
            assert pt.selected_variant(m, n, k, ta, tb) in kappa
        X = matrix("normal", 4, M, K, std=0.02)
        W = matrix("normal", 5, K, N, std=0.02)
        G = matrix("normal", 6, M, N)
        Xd = torch.from_numpy(X).cuda().requires_grad_(True)
        Wd = torch.from_numpy(W).cuda().requires_grad_(True)
        Y = matmul(Xd, Wd)
        Y.backward(torch.from_numpy(G).cuda())
        torch.cuda.synchronize()
        rows = [0, 1, 777, 2048, 4095]
        assert normalised_error(Y.detach()[rows].cpu().numpy(), og.gemm(X, W, rows=rows), K,
                                np.abs(X).max(), np.abs(W).max()) <= TOL_FP32
        assert normalised_error(Xd.grad[rows].cpu().numpy(), og.gemm(G, W, "N", "T", rows=rows), N,
                                np.abs(G).max(), np.abs(W).max()) <= TOL_FP32
        wrows = [0, 511, 1023]
        assert normalised_error(Wd.grad[wrows].cpu().numpy(), og.gemm(X, G, "T", "N", rows=wrows), M,
                                np.abs(X).max(), np.abs(G).max()) <= TOL_FP32
    finally:
        pt.load_manifest(None)
