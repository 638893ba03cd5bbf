"""GPU: the kernel timer records one event pair per GEMM call around the
main kernel only, and nothing for calls captured into a CUDA graph."""

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"


def _inputs(M, N, K):
    g = torch.Generator(device="cpu").manual_seed(7)
    A = (torch.rand((M, K), generator=g) * 2 - 1).to(DEV)
    B = (torch.rand((K, N), generator=g) * 2 - 1).to(DEV)
    return A, B, torch.empty((M, N), device=DEV)


@pytest.mark.parametrize("name", ["tcbf16x3_m128n128_p2", "tc3xtf32_m128n128_p3", None])
def test_timer_counts_main_kernels(name):
    M = N = K = 1024
    A, B, C = _inputs(M, N, K)
    vid = pt.default_variant() if name is None else pt.variant_by_name(name)
    s = torch.cuda.Stream(DEV)
    with torch.cuda.stream(s):
        pt.sgemm(A, B, C, variant=vid, stream=s)
        s.synchronize()
        pt.kernel_timer_start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(5):
            pt.sgemm(A, B, C, variant=vid, stream=s)
        e1.record(s)
        ms, n = pt.kernel_timer_stop()
    s.synchronize()
    assert n == 5
    call_ms = e0.elapsed_time(e1)
    assert 0.0 < ms <= call_ms * 1.05
    if pt.variant(vid)["kind"] != 0:
        # The split kernel is outside the timed interval.
        assert ms < call_ms


def test_timer_ignores_captured_calls():
    A, B, C = _inputs(512, 512, 512)
    s = torch.cuda.Stream(DEV)
    with torch.cuda.stream(s):
        pt.sgemm(A, B, C, stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        pt.kernel_timer_start()
        with torch.cuda.graph(g, stream=s):
            pt.sgemm(A, B, C, stream=s)
        ms, n = pt.kernel_timer_stop()
        g.replay()
    s.synchronize()
    assert (ms, n) == (0.0, 0)
    assert pt.device_status() == 0
