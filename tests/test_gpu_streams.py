"""GPU: calls on two streams at once.  Each stream has its own split-plane
workspace (and stream-K flags), so tensor-core calls issued concurrently on
two streams must not interfere; results are compared with the oracle."""

import numpy as np
import pytest

from oracle import gemm as og
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
NAMES = ["tcbf16x3_m128n128_p4_sw64_stk", "tcbf16x3_m128n128_p2", "tc3xtf32_m128n128_p3_stk",
         "tcbf16x3_m128n64_p2_fb_sk2"]


@pytest.mark.parametrize("first,second", [(NAMES[0], NAMES[0]), (NAMES[0], NAMES[1]), (NAMES[2], NAMES[3])])
def test_two_streams_concurrent_tensor_core_calls(first, second):
    shapes = [(1024, 1024, 4096), (768, 1280, 2048)]
    data = []
    for i, (M, N, K) in enumerate(shapes):
        A = matrix("ints", 70 + i, M, K)
        B = matrix("ints", 80 + i, K, N)
        data.append((A, B, og.gemm(A, B, M=M, N=N, K=K)))
    s0, s1 = torch.cuda.Stream(DEV), torch.cuda.Stream(DEV)
    dev = [(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)) for A, B, _ in data]
    outs = [[torch.empty((M, N), device=DEV) for _ in range(6)] for (M, N, K) in shapes]
    torch.cuda.synchronize()
    vids = [pt.variant_by_name(first), pt.variant_by_name(second)]
    for rep in range(6):  # interleaved issue: the two streams' kernels overlap on the GPU
        for j, s in enumerate((s0, s1)):
            with torch.cuda.stream(s):
                pt.sgemm(dev[j][0], dev[j][1], outs[j][rep], variant=vids[j], stream=s)
    torch.cuda.synchronize()
    for j in range(2):
        for rep in range(6):
            assert np.array_equal(outs[j][rep].cpu().numpy().astype(np.float64), data[j][2]), (j, rep)
    assert pt.device_status() == 0
