"""GPU parity: every variant of the family against the FP64 CPU oracle.

Bit-exact on small-integer inputs (all partial sums are integers below 2^24,
so any summation order gives the exact result); within the normalised error
bound 2e-6 on uniform and log-uniform inputs.
"""

import numpy as np
import pytest

from oracle import gemm as og
from oracle.checks import TOL_FP32, normalised_error
from workloads import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

DEV = "cuda:0"
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]
_cache = {}


def _store(X, t, align=1):
    """Row-major storage of op^-1(X); leading dimension rounded up to `align`
    with NaN padding (never read by a correct kernel)."""
    S = np.ascontiguousarray(X.T if t == "T" else X)
    ld = -(-S.shape[1] // align) * align
    if ld == S.shape[1]:
        return S
    P = np.full((S.shape[0], ld), np.nan, np.float32)
    P[:, :S.shape[1]] = S
    return P


def _case(kind, M, N, K, ta, tb, seed, align=4):
    key = (kind, M, N, K, ta, tb, seed, align)
    if key not in _cache:
        A = matrix(kind, seed, M, K)
        B = matrix(kind, seed + 1, K, N)
        As, Bs = _store(A, ta, align), _store(B, tb, align)
        ref = og.gemm(As, Bs, ta, tb, M=M, N=N, K=K)
        _cache[key] = (As, Bs, ref, float(np.abs(A).max()), float(np.abs(B).max()))
    return _cache[key]


def _supports(desc, ta, tb):
    return bool(desc["trans_mask"] >> ((ta == "T") * 2 + (tb == "T")) & 1)


def _run(vid, As, Bs, M, N, ta, tb, alpha=1.0, beta=0.0, C0=None, K=None, may_decline=False):
    """Runs variant `vid` (None: pt_sgemm) on padded storage; returns C (M x N),
    or None when `may_decline` and the variant's admission rules refuse the
    arguments (PT_EUNSUPPORTED, nothing launched)."""
    if K is None:
        K = As.shape[1] if ta == "N" else As.shape[0]
    Ad = torch.from_numpy(As).to(DEV)
    Bd = torch.from_numpy(Bs).to(DEV)
    Al = Ad[:M, :K] if ta == "N" else Ad[:K, :M]
    Bl = Bd[:K, :N] if tb == "N" else Bd[:N, :K]
    ldc = -(-N // 4) * 4
    store = torch.full((M, ldc), float("nan"), device=DEV)  # every output must be written
    Cd = store[:, :N]
    if C0 is not None:
        Cd.copy_(torch.from_numpy(C0).to(DEV))
    try:
        pt.sgemm(Al, Bl, Cd, ta, tb, alpha, beta, variant=vid)
    except pt.PtError as e:
        if may_decline and e.code == -2:
            return None
        raise
    torch.cuda.synchronize()
    return Cd.cpu().numpy()


NVAR = None


def _nvar():
    global NVAR
    if NVAR is None:
        NVAR = pt.num_variants()
    return NVAR


SMALL_SHAPES = [(131, 97, 75), (33, 260, 19)]


@pytest.mark.parametrize("vid", range(456))
def test_variant_bit_exact_small_integers(vid):
    if vid >= _nvar():
        pytest.skip("registry has fewer variants")
    d = pt.variant(vid)
    ran = 0
    for (M, N, K) in SMALL_SHAPES:
        for ta, tb in TRANS:
            if not _supports(d, ta, tb):
                continue
            As, Bs, ref, _, _ = _case("ints", M, N, K, ta, tb, 11)
            out = _run(vid, As, Bs, M, N, ta, tb, K=K)
            assert np.array_equal(out.astype(np.float64), ref), (d["name"], M, N, K, ta, tb)
            ran += 1
    assert ran > 0


@pytest.mark.parametrize("vid", range(456))
def test_variant_uniform_within_bound(vid):
    if vid >= _nvar():
        pytest.skip("registry has fewer variants")
    d = pt.variant(vid)
    M, N, K = 300, 200, 1000
    ta, tb = ("T", "N") if d["trans_mask"] == 4 else ("N", "N")
    As, Bs, ref, ma, mb = _case("uniform", M, N, K, ta, tb, 21)
    out = _run(vid, As, Bs, M, N, ta, tb, K=K)
    err = normalised_error(out, ref, K, ma, mb)
    assert err <= TOL_FP32, (d["name"], err)


def test_alpha_beta_and_nan_c():
    M, N, K = 150, 130, 70
    A = matrix("uniform", 5, M, K)
    B = matrix("uniform", 6, K, N)
    C0 = matrix("uniform", 7, M, N)
    ref = og.gemm(A, B, alpha=1.5, beta=-0.5, C=C0)
    for vid in range(0, _nvar(), 7):
        if not _supports(pt.variant(vid), "N", "N"):
            continue
        out = _run(vid, A, B, M, N, "N", "N", 1.5, -0.5, C0, may_decline=True)
        if out is None:
            continue
        err = normalised_error(out, ref, K, np.abs(A).max(), np.abs(B).max(), 1.5, -0.5, np.abs(C0).max())
        assert err <= TOL_FP32, (vid, err)
    # beta = 0: NaN already in C must not propagate.
    out = _run(0, A, B, M, N, "N", "N", 2.0, 0.0, np.full((M, N), np.nan, np.float32))
    assert np.all(np.isfinite(out))


@pytest.mark.parametrize("N,ldc", [(90, 96), (92, 100)])  # N % 4 == 0: tensor-core versions store C by TMA
def test_padded_leading_dimensions_and_canary(N, ldc):
    M, K = 77, 45
    lda, ldb = 52, 100
    A = matrix("ints", 31, M, K, ld=lda)        # padding columns are NaN
    B = matrix("ints", 32, K, N, ld=ldb)
    ref = og.gemm(A, B, K=K, N=N)
    canary = np.float32(12345.0)
    for vid in range(0, _nvar(), 5):
        Ad = torch.from_numpy(A).to(DEV)
        Bd = torch.from_numpy(B).to(DEV)
        store = torch.full((M + 32, ldc), float(canary), device=DEV)  # guard rows: a box's height
        Cd = store[:M, :N]
        try:
            pt.sgemm(Ad[:, :K], Bd[:, :N], Cd, variant=vid)
        except pt.PtError as e:
            assert e.code == -2  # alignment/layout admission only
            continue
        torch.cuda.synchronize()
        full = store.cpu().numpy()
        assert np.array_equal(full[:M, :N].astype(np.float64), ref), vid
        assert np.all(full[:M, N:] == canary) and np.all(full[M:] == canary), vid


def test_default_variant_runs_every_layout_and_alignment():
    M, N, K = 45, 37, 29
    for ta, tb in TRANS:
        As, Bs, ref, _, _ = _case("ints", M, N, K, ta, tb, 41, align=1)
        # odd leading dimensions defeat vector loads; the default variant still runs
        out = _run(pt.default_variant(), As, Bs, M, N, ta, tb, K=K)
        assert np.array_equal(out.astype(np.float64), ref)
        out = _run(None, As, Bs, M, N, ta, tb, K=K)
        assert np.array_equal(out.astype(np.float64), ref)


def test_config_256_fixed_variant():
    vid = pt.variant_by_name("s128x128x8_w32x64_t8x8_kl1_v4_p2_sk1_cpm")
    A = matrix("uniform", 1, 256, 256)
    B = matrix("uniform", 2, 256, 256)
    ref = og.gemm(A, B)
    out = _run(vid, A, B, 256, 256, "N", "N")
    err = normalised_error(out, ref, 256, np.abs(A).max(), np.abs(B).max())
    assert err <= TOL_FP32, err


@pytest.mark.parametrize("name_part", ["sk1_cpm", "sk4_cpk", "tmk", "kl2", "sk8", "tc3xtf32", "tcbf16x3"])
def test_full_size_sampled_rows(name_part):
    """4096^3 (largest sweep shape) on sampled rows, inputs U[-1,1]."""
    M = N = K = 4096
    cands = [v for v in pt.variants() if name_part in v["name"] and v["trans_mask"] & 1]
    assert cands, name_part
    vid = cands[0]["id"]
    A = matrix("uniform", 1000 + 63, M, K)
    B = matrix("uniform", 1000 + 64, K, N)
    rows = np.sort(np.random.default_rng(0).choice(M, 48, replace=False))
    ref = og.gemm(A, B, rows=rows)
    out = _run(vid, A, B, M, N, "N", "N")[rows]
    err = normalised_error(out, ref, K, np.abs(A).max(), np.abs(B).max())
    assert err <= TOL_FP32, (cands[0]["name"], err)


def test_log_uniform_magnitudes():
    M, N, K = 256, 192, 512
    A = matrix("logu", 3, M, K)
    B = matrix("logu", 4, K, N)
    ref = og.gemm(A, B)
    for vid in range(0, _nvar(), 11):
        if not _supports(pt.variant(vid), "N", "N"):
            continue
        out = _run(vid, A, B, M, N, "N", "N", may_decline=True)
        if out is None:
            continue
        err = normalised_error(out, ref, K, np.abs(A).max(), np.abs(B).max())
        assert err <= TOL_FP32, (vid, err)


def test_quick_returns():
    A = torch.ones((4, 0), device=DEV)
    B = torch.ones((0, 3), device=DEV)
    C = torch.full((4, 3), 2.0, device=DEV)
    pt.sgemm(A, B, C, beta=0.5)               # K = 0: C <- beta*C
    torch.cuda.synchronize()
    assert torch.all(C == 1.0)
    A = torch.ones((4, 5), device=DEV)
    B = torch.ones((5, 3), device=DEV)
    pt.sgemm(A, B, C, alpha=0.0, beta=0.0)    # alpha = 0, beta = 0: C <- 0
    torch.cuda.synchronize()
    assert torch.all(C == 0.0)
    E = torch.empty((0, 3), device=DEV)
    pt.sgemm(torch.ones((0, 5), device=DEV), B, E)  # M = 0: nothing to do


def test_reference_kernel_close_to_oracle():
    M, N, K = 200, 150, 2000
    A = matrix("uniform", 51, M, K)
    B = matrix("uniform", 52, K, N)
    ref = og.gemm(A, B)
    out = pt.reference(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)).cpu().numpy()
    err = normalised_error(out, ref, K, np.abs(A).max(), np.abs(B).max())
    assert err <= 1e-7, err  # compensated dot: about one FP32 rounding of the result


def test_split_k_is_deterministic():
    cands = [v["id"] for v in pt.variants() if v["splitk"] > 1 and v["trans_mask"] & 1]
    A = torch.from_numpy(matrix("uniform", 61, 200, 3000)).to(DEV)
    B = torch.from_numpy(matrix("uniform", 62, 3000, 192)).to(DEV)
    for vid in cands[:6]:
        c1 = pt.sgemm(A, B, variant=vid)
        c2 = pt.sgemm(A, B, variant=vid)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2), vid


def test_argument_errors():
    A = torch.ones((4, 4), device=DEV)
    B = torch.ones((4, 3), device=DEV)
    C = torch.empty((4, 3), device=DEV)
    with pytest.raises(pt.PtError) as e:
        pt.sgemm(A, B, C, transA="X")
    assert e.value.code == -1 and e.value.arg == 1
    tma = [v["id"] for v in pt.variants() if v["loader"] == 1 and v["a_kmajor"]]
    with pytest.raises(pt.PtError) as e:
        pt.sgemm(A, B, C, transA="T", variant=tma[0])
    assert e.value.code == -2
    assert pt.device_status() == 0
