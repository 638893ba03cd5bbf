"""GPU: the sweep in the launch configuration the benchmark times.  All 64
shapes of the {128, 512, 1024, 4096}^3 sweep run through pt_sgemm with a
loaded manifest whose members cover every family a selection deploys (SIMT,
persistent, cluster split-K, stream-K, fused-A and fused-B tensor-core
versions).  The 64 calls are captured once as a CUDA graph, on one stream
and one split workspace shared by consecutive calls, and replayed twice with
every output NaN-poisoned in between.  Inputs are the benchmark's (U[-1,1],
A seed 1000 + i, B seed 101000 + i for shape i); each output is checked
against the FP64 oracle on sampled rows."""

import json

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix, sweep_shapes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
KAPPA = ["s32x32x16_w16x16_t4x4_kl2_v4_p3_sk4_cpk", "tcbf16x3_m128n128_p2", "tcbf16x3_m128n64_p3_sk8",
         "tcbf16x3_m128n128_p4_sw64_stk", "tcbf16x3_m128n128_p3_sw64_fa_sk4", "tcbf16x3_m128n128_p3_sw64_fb_sk4",
         "tcbf16x3_m128n64_p2", "tcbf16x3_m128n64_p2_sk4"]
ROWS = 6  # sampled rows per shape


def _manifest(path, shapes):
    # Shape i is listed with member i mod 8, so that every member runs shapes
    # of every size class; a listed shape takes its member exactly.
    entries = [{"m": M, "n": N, "k": K, "transA": "N", "transB": "N", "variant": KAPPA[i % len(KAPPA)]}
               for i, (M, N, K) in enumerate(shapes)]
    with open(path, "w") as f:
        json.dump({"format": "pt-manifest-1", "method": "fixed", "k": len(KAPPA), "train_geomean": 1.0,
                   "kappa": KAPPA, "map": entries}, f)


def test_sweep_graph_through_manifest(tmp_path):
    shapes = sweep_shapes()
    assert len(shapes) == 64
    man = str(tmp_path / "kappa.json")
    _manifest(man, shapes)
    A = [matrix("uniform", 1000 + i, M, K) for i, (M, N, K) in enumerate(shapes)]
    B = [matrix("uniform", 101000 + i, K, N) for i, (M, N, K) in enumerate(shapes)]
    Ad = [torch.from_numpy(a).to(DEV) for a in A]
    Bd = [torch.from_numpy(b).to(DEV) for b in B]
    Cd = [torch.empty((M, N), device=DEV) for (M, N, K) in shapes]
    pt.load_manifest(man)
    try:
        for i, (M, N, K) in enumerate(shapes):
            assert pt.selected_variant(M, N, K, A=Ad[i], B=Bd[i], C=Cd[i]) == \
                pt.variant_by_name(KAPPA[i % len(KAPPA)]), shapes[i]
        s = torch.cuda.Stream(DEV)

        def step():
            for i in range(len(shapes)):
                pt.sgemm(Ad[i], Bd[i], Cd[i], stream=s)

        with torch.cuda.stream(s):
            step()  # workspace and attributes set up outside the capture
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                step()
        for _ in range(2):
            for c in Cd:
                c.fill_(float("nan"))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            for i, (M, N, K) in enumerate(shapes):
                rows = np.unique(np.linspace(0, M - 1, ROWS).astype(np.int64))
                ref = og.gemm(A[i], B[i], rows=rows)
                got = Cd[i][torch.from_numpy(rows).to(DEV)].cpu().numpy()
                e = normalised_error(got, ref, K, np.abs(A[i]).max(), np.abs(B[i]).max())
                assert e <= TOL_FP32, (shapes[i], KAPPA[i % len(KAPPA)], e)
        assert pt.device_status() == 0
    finally:
        pt.load_manifest(None)
