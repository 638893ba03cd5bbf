"""GPU: stream-K tensor-core versions.  Tiles shared by several CTAs are
finished by the CTA that owns their last chunk, which adds the partial tiles
the others publish through the workspace (flags carry a per-launch epoch).
Shapes are chosen so that tiles are split across two CTAs, across many CTAs
(one 128-k chunk each), and within a single CTA's range; results must be
bit-exact on small integers, within the FP32 bound on uniform inputs, and
stay so over repeated launches and graph replays (the epoch advances)."""

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
STK = ["tcbf16x3_m128n128_p2_stk", "tcbf16x3_m128n128_p4_sw64_stk", "tcbf16x3_m128n64_p3_stk",
       "tc3xtf32_m128n128_p3_stk", "tc3xtf32_m128n64_p4_stk", "tc3xf16_m128n128_p3_stk",
       "tc3xf16_m128n256_p4_sw64_stk", "tc3xf16_m256n256_p6_sw64_2sm_stk"]
SHAPES = [(1024, 1024, 4096),   # 64 or 128 tiles x 32 chunks over the SMs: tiles split between CTAs
          (256, 256, 4096),     # few tiles, one chunk per CTA: many contributors per tile
          (300, 200, 1000),     # ragged edges, 8 chunks per tile
          (640, 384, 2176)]     # ragged chunk count (17)
_cache = {}


def _ref(kind, M, N, K):
    key = (kind, M, N, K)
    if key not in _cache:
        A = matrix(kind, 21, M, K)
        B = matrix(kind, 22, K, N)
        _cache[key] = (A, B, og.gemm(A, B, M=M, N=N, K=K), float(np.abs(A).max()), float(np.abs(B).max()))
    return _cache[key]


@pytest.mark.parametrize("name", STK)
@pytest.mark.parametrize("shape", SHAPES)
def test_streamk_exact_on_integers(name, shape):
    M, N, K = shape
    A, B, ref, _, _ = _ref("ints", M, N, K)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.full((M, N), float("nan"), device=DEV)
    vid = pt.variant_by_name(name)
    for _ in range(3):  # repeated launches: later ones must not read earlier partials
        C.fill_(float("nan"))
        pt.sgemm(Ad, Bd, C, variant=vid)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
    assert pt.device_status() == 0


@pytest.mark.parametrize("name", STK[:2] + STK[3:4])
def test_streamk_uniform_and_graph_replay(name):
    M, N, K = 1024, 1024, 4096
    A, B, ref, amax, bmax = _ref("uniform", M, N, K)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.empty((M, N), device=DEV)
    vid = pt.variant_by_name(name)
    s = torch.cuda.Stream(DEV)
    with torch.cuda.stream(s):
        pt.sgemm(Ad, Bd, C, variant=vid, stream=s)  # workspace set-up outside the capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            pt.sgemm(Ad, Bd, C, variant=vid, stream=s)
        for _ in range(4):
            C.fill_(float("nan"))
            g.replay()
            s.synchronize()
            e = normalised_error(C.cpu().numpy(), ref, K, amax, bmax)
            assert e <= TOL_FP32
    assert pt.device_status() == 0


def test_streamk_alpha_beta():
    M, N, K = 512, 768, 3072
    A, B, _, amax, bmax = _ref("uniform", M, N, K)
    C0 = matrix("uniform", 23, M, N)
    ref = og.gemm(A, B, alpha=0.75, beta=-1.25, C=C0, M=M, N=N, K=K)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    for name in STK:
        C = torch.from_numpy(C0.copy()).to(DEV)
        pt.sgemm(Ad, Bd, C, alpha=0.75, beta=-1.25, variant=pt.variant_by_name(name))
        torch.cuda.synchronize()
        e = normalised_error(C.cpu().numpy(), ref, K, amax, bmax, alpha=0.75, beta=-1.25,
                             maxC=float(np.abs(C0).max()))
        assert e <= TOL_FP32, name


def test_streamk_after_shutdown_recreates_workspace():
    # pt_shutdown frees the workspaces (and their stream-K flags); the next
    # call allocates a fresh, zeroed one and must still be exact.
    M, N, K = 1024, 1024, 4096
    A, B, ref, _, _ = _ref("ints", M, N, K)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    vid = pt.variant_by_name(STK[0])
    for _ in range(2):
        C = pt.sgemm(Ad, Bd, variant=vid)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
        pt.shutdown()


@pytest.mark.parametrize("name", STK)
def test_streamk_whole_tiles_near_one_wave(name):
    # Between 3/4 of a wave and a wave of tiles the launcher gives each tile
    # its own CTA (no shared tiles); the result is the same exact integer.
    d = pt.variant(pt.variant_by_name(name))
    sms = torch.cuda.get_device_properties(DEV).multi_processor_count
    rows = 12
    cols = (sms * 9 // 10) // rows  # 0.9 of a wave of tiles
    M, N, K = rows * d["bm"], cols * d["bn"], 520
    A = matrix("ints", 23, M, K)
    B = matrix("ints", 24, K, N)
    ref = og.gemm(A, B)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.full((M, N), float("nan"), device=DEV)
    vid = pt.variant_by_name(name)
    for _ in range(2):
        C.fill_(float("nan"))
        pt.sgemm(Ad, Bd, C, variant=vid)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.float64), ref), (name, M, N, K)
    assert pt.device_status() == 0


@pytest.mark.parametrize("tiles_over", [10, -20])
def test_hybrid_wide_version_both_schedules(tiles_over):
    # tc3xf16_m128n256_p4_sw64 runs its stream-K twin when the tiles make more
    # than a wave with a last wave under 3/4 full (tiles_over = 10), one CTA per
    # tile otherwise (tiles_over = -20); both give the exact integer result.
    name = "tc3xf16_m128n256_p4_sw64"
    sms = torch.cuda.get_device_properties(DEV).multi_processor_count
    rows = 12
    cols = (sms + tiles_over) // rows + 1
    M, N, K = rows * 128, cols * 256, 520
    A = matrix("ints", 25, M, K)
    B = matrix("ints", 26, K, N)
    ref = og.gemm(A, B)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.full((M, N), float("nan"), device=DEV)
    for _ in range(2):
        C.fill_(float("nan"))
        pt.sgemm(Ad, Bd, C, variant=pt.variant_by_name(name))
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.float64), ref), (M, N, K)
    assert pt.device_status() == 0
