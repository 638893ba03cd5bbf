"""GPU: failure paths, made on the host or by a bounded wait that runs out.

* Data collection (the paper's Section V-D screens out kernels that fail and
  keeps collecting): the tuner's fail_launch hook makes one variant launch
  report an error without launching anything.  That row must be recorded
  invalid with the error as its status, and every other row must still be
  measured.
* Stream-K hand-over: with pt_debug_streamk_wait(limit, never_ready=1) the
  CTAs that finish shared tiles wait for a flag value nobody writes; after
  the limit (1 ms here) each skips its tile's stores and the kernel ends.
  The call must then be reported by pt_device_status as PT_ETIMEOUT, the
  tiles nobody shares must still be right, and once the hook is off the next
  launch on the same workspace must be exact again.  Nothing faults, traps or
  hangs: the kernel's other waits keep their normal limit, and the timed-out
  wait is the last thing a finishing CTA does, after all of its tensor-core
  work and copies have completed.
"""

import csv

import numpy as np
import pytest

from oracle import gemm as og
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"


def _rows(path):
    with open(path) as f:
        return list(csv.DictReader(f))


@pytest.mark.parametrize("fail_at", [1, 5])
def test_tuner_records_failed_launch_and_continues(tmp_path, fail_at):
    # fail_at 1: the first variant's screening launch; 5: one of its timed launches
    path = str(tmp_path / "t.csv")
    ids = [pt.default_variant(), pt.variant_by_name("tc3xtf32_m128n128_p3"),
           pt.variant_by_name("tcbf16x3_m128n128_p2_stk")]
    shapes = [(256, 256, 512), (384, 128, 1024)]
    pt.tune(shapes, path, ids=ids, reps_min=3, reps_max=5, target_ms=0.5, warmup=2, fail_launch=fail_at)
    rows = _rows(path)
    assert len(rows) == len(ids) * len(shapes)
    first = rows[0]
    assert first["variant"] == pt.variant(ids[0])["name"]
    assert int(first["valid"]) == 0 and int(first["status"]) == pt._lib.PT_ECUDA
    for r in rows[1:]:
        assert int(r["valid"]) == 1 and int(r["status"]) == 0, r
        assert float(r["median_ms"]) > 0
    assert pt.device_status() == 0


def test_streamk_wait_that_runs_out_reports_timeout_and_recovers():
    name = "tcbf16x3_m128n128_p2_stk"
    vid = pt.variant_by_name(name)
    # 32 x 12 tiles of 128 x 128 and 4 chunks of k: a first wave of whole tiles,
    # then the remaining tiles' chunks shared out, most tiles between two CTAs
    M, N, K = 4096, 1536, 512
    A = matrix("ints", 71, M, K)
    B = matrix("ints", 72, K, N)
    ref = og.gemm(A, B)
    Ad, Bd = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    C = torch.full((M, N), float("nan"), device=DEV)
    pt.sgemm(Ad, Bd, C, variant=vid)           # workspace set up, flags at a valid epoch
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
    assert pt.device_status() == 0
    try:
        pt.debug_streamk_wait(1_000_000, never_ready=True)
        C.fill_(float("nan"))
        pt.sgemm(Ad, Bd, C, variant=vid)
        torch.cuda.synchronize()
        assert pt.device_status() == pt._lib.PT_ETIMEOUT
    finally:
        pt.debug_streamk_wait(0, never_ready=False)
    out = C.cpu().numpy().astype(np.float64)
    written = ~np.isnan(out)
    assert 0 < written.sum() < out.size            # finished tiles were skipped, the rest stored
    assert np.array_equal(out[written], ref[written])
    assert pt.device_status() == 0                  # reading cleared the word
    for _ in range(2):                              # later launches: epochs still line up
        C.fill_(float("nan"))
        pt.sgemm(Ad, Bd, C, variant=vid)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
    assert pt.device_status() == 0
