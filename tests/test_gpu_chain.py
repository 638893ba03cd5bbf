"""GPU: dependent launches in one stream.  The SIMT, split and tensor-core
kernels are launched with programmatic stream serialization, so each must wait
for its predecessor before touching memory.  A chain of GEMMs whose every
input is the previous output (outputs NaN-poisoned beforehand) checks that no
kernel reads or overwrites data early: the results are exact integers and
must equal the oracle bit for bit, eagerly and replayed from a CUDA graph."""

import numpy as np
import pytest

from oracle import gemm as og
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
# (variant names, alternating families); the first GEMM is long (K = 4096).
CHAINS = [
    ["s128x128x8_w32x64_t8x8_kl1_v1_p2_sk1_cpm", "tcbf16x3_m128n128_p2", "tc3xtf32_m128n128_p3",
     "s128x128x8_w32x64_t8x8_kl1_v1_p2_sk1_cpm"],
    ["tcbf16x3_m128n128_p4_sw64", "tc3xtf32_m128n64_p4_sk4", "tcbf16x3_m128n64_p3", "tcbf16x3_m128n128_p2_sk2"],
    # fused split and stream-K: a fused-A GEMM reads its predecessor's output itself
    ["tcbf16x3_m128n128_p3_sw64_fa_sk4", "tcbf16x3_m128n128_p4_sw64_stk", "tcbf16x3_m128n128_p3_sw64_fb_stk",
     "tcbf16x3_m128n64_p3_sw64_fa_stk"],
]


def _signed_permutation(n, seed):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, n), np.float32)
    P[np.arange(n), rng.permutation(n)] = rng.choice([-1.0, 1.0], n).astype(np.float32)
    return P


_cache = {}


def _expected(A, B, P, steps):
    if steps in _cache:
        return _cache[steps]
    X = og.gemm(A, B, "N", "N", M=A.shape[0], N=B.shape[1], K=A.shape[1])
    out = [X]
    for _ in range(steps - 1):
        X = og.gemm(X.astype(np.float32), P, "N", "N", M=X.shape[0], N=P.shape[1], K=P.shape[0])
        out.append(X)
    _cache[steps] = out
    return out


@pytest.mark.parametrize("chain", range(len(CHAINS)))
@pytest.mark.parametrize("graph", [False, True])
def test_dependent_chain_is_exact(chain, graph):
    names = CHAINS[chain]
    M, K, N = 1024, 4096, 1024
    A = matrix("ints", 11, M, K)
    B = matrix("ints", 12, K, N)
    P = _signed_permutation(N, 13)
    expect = _expected(A, B, P, len(names))
    # Integer partial sums below 2^22: exact in FP32, in the TF32 hi+lo split
    # and in the BF16 triple split.
    assert max(np.abs(e).max() for e in expect) < 2 ** 22
    ids = [pt.variant_by_name(n) for n in names]
    Ad, Bd, Pd = (torch.from_numpy(x).to(DEV) for x in (A, B, P))
    outs = [torch.empty((M, N), device=DEV) for _ in names]
    s = torch.cuda.Stream(DEV)

    def run():
        src = Ad
        for i, vid in enumerate(ids):
            pt.sgemm(src, Bd if i == 0 else Pd, outs[i], variant=vid, stream=s)
            src = outs[i]

    with torch.cuda.stream(s):
        if graph:
            run()  # workspace set-up outside the capture
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                run()
            for o in outs:
                o.fill_(float("nan"))
            g.replay()
        else:
            for o in outs:
                o.fill_(float("nan"))
            run()
    s.synchronize()
    for i, (o, e) in enumerate(zip(outs, expect)):
        got = o.cpu().numpy().astype(np.float64)
        assert np.array_equal(got, e), "step %d (%s) differs" % (i, names[i])
    assert pt.device_status() == 0
