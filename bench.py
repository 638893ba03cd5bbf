"""Benchmark: portability-tuned SGEMM on the 64-shape sweep.

One step = one pass of the hot path over the sweep workload: every
(M, N, K) in {128, 512, 1024, 4096}^3 (FP32 row-major, alpha=1, beta=0,
inputs U[-1,1] from SplitMix64 with seed 1000 + shape index) through the
multi-versioned entry point pt_sgemm, whose runtime selector picks one of
the k = 8 variants chosen by PortabilityTune on the training half of the
shapes (the other half is held out).  Before the timed region the bench
runs the data collection (timing table of every variant on every shape) and
the selection (k = 1..8); their results are reported alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Output: one JSON line on rank 0.  `value` is whole-job SGEMM TFLOP/s with
inputs resident in HBM (1.6 GB of inputs, larger than L2); `e2e` adds the
per-step host->device copies of A and B and the device->host copy of C.
Multi-GPU: independent replicas (one per rank), weak scaling; no collective
on the data path.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SGEMM TFLOP/s per shape; geomean % of per-shape best variant using k selected"
UNIT = "TFLOP/s"
WORKLOAD = "portability sweep: (M,N,K) in {128,512,1024,4096}^3, 64 shapes, FP32 row-major NN, alpha=1, beta=0, U[-1,1]"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--k", type=int, default=8, help="size of the deployed variant set")
    p.add_argument("--table", default=None, help="reuse an existing timing table")
    p.add_argument("--out-dir", default=None, help="where the table and manifests are written")
    p.add_argument("--tune-reps-max", type=int, default=30)
    p.add_argument("--tune-target-ms", type=float, default=3.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-rows", type=int, default=512, help="rows per shape in the CPU-oracle sample")
    p.add_argument("--single", default=None, metavar="M,N,K",
                   help="profiling mode: run one variant (--variant) on one shape, no tuning")
    p.add_argument("--variant", default=None, help="variant name for --single")
    p.add_argument("--report", default=None,
                   choices=["splitprec", "grouped", "stability", "oracle", "autograd", "noalloc"],
                   help="splitprec: tensor-core split-precision vs FP32 SIMT on the split-precision shapes; "
                        "grouped: 512 uneven problems, persistent grouped launch vs separate launches; "
                        "stability: the sweep tuned twice, rank agreement of the two timing tables; "
                        "oracle: the FP64 CPU oracle timed at 256^3, 1024^3 and 4096^3; "
                        "autograd: Y = X W forward and backward through the tuned SGEMM; "
                        "noalloc: the allocation-free entry point against its registry twin")
    return p.parse_args()


def report_grouped(args):
    """512 independent problems (M, N, K = 8*round(2^U[5,11]/8), clamped to
    [32, 2048], seed 5; entries U[-1,1]): one persistent grouped launch with
    per-problem tiles from the k = 8 selector, against 512 separate launches
    of the single best variant (k = 1) and 512 pt_sgemm calls through the
    k = 8 selector.  Every arm is captured once as a CUDA graph and replayed;
    CUDA-event time over the replays."""
    import torch

    import paper_2507_15277_gb300 as pt
    from workloads import grouped_problems, matrix, parity_split, sweep_shapes
    dev = torch.device("cuda", 0)
    out_dir = args.out_dir or tempfile.mkdtemp(prefix="ptgrouped_")
    os.makedirs(out_dir, exist_ok=True)
    table = args.table or os.path.join(out_dir, "table.csv")
    if not args.table:
        pt.tune(sweep_shapes(), table, reps_min=5, reps_max=args.tune_reps_max, target_ms=args.tune_target_ms)
    train, _ = parity_split()
    m1, m8 = os.path.join(out_dir, "grouped_k1.json"), os.path.join(out_dir, "grouped_k8.json")
    ids1, _ = pt.select(table, train, 1, manifest=m1)
    pt.select(table, train, 8, manifest=m8)
    probs = grouped_problems()
    items = []
    for i, (M, N, K) in enumerate(probs):
        A = torch.from_numpy(matrix("uniform", 5000 + i, M, K)).to(dev)
        B = torch.from_numpy(matrix("uniform", 6000 + i, K, N)).to(dev)
        items.append((A, B, torch.empty((M, N), device=dev), "N", "N", 1.0, 0.0))
    flops = sum(2.0 * M * N * K for (M, N, K) in probs)
    pt.load_manifest(m8)
    arr = pt.grouped_problems(items)
    ddesc = pt.upload_problems(arr, dev)
    tiles = {}
    for i in range(len(items)):
        tiles[arr[i].tile] = tiles.get(arr[i].tile, 0) + 1
    stream = torch.cuda.Stream(dev)

    def arm_single():
        for (A, B, C, *_r) in items:
            pt.sgemm(A, B, C, variant=ids1[0], stream=stream)

    def arm_selector():
        for (A, B, C, *_r) in items:
            pt.sgemm(A, B, C, stream=stream)

    def arm_grouped():
        pt.sgemm_grouped(arr, ddesc=ddesc, stream=stream, device=dev)

    res = {}
    reps = max(3, args.steps // 10)
    for name, fn in (("single_best_512_launches", arm_single), ("selector_512_launches", arm_selector),
                     ("grouped_persistent_1_launch", arm_grouped)):
        with torch.cuda.stream(stream):
            fn()  # warm: attributes, workspaces
            stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                fn()
            for _ in range(3):
                g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
            stream.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12}
        del g
    pt.load_manifest(None)
    print(json.dumps({"mode": "grouped", "problems": len(probs), "gflop": flops / 1e9,
                      "single_best_variant": pt.variant(ids1[0])["name"], "tiles_used": tiles,
                      "replays": reps, "arms": res}))
    return 0


def report_splitprec(args):
    """Split-precision tensor-core variants vs the FP32 SIMT family on
    M=N=K in {1024, 4096, 8192}, 8192x8192x256 and 256x8192x8192, inputs of
    random sign with magnitudes 2^U[-10,10] (seed 3): TFLOP/s of the fastest
    variant of each kind (timed by the tuner, split kernel included) and the
    measured TF32 cuBLAS throughput at 8192^3 as the TF32 reference.  The
    error of every one of these variants against the FP64 oracle on these
    inputs is measured by tests/test_gpu_config3.py (PT_PARITY_REPORT)."""
    import torch

    import paper_2507_15277_gb300 as pt
    from workloads import split_precision_shapes
    dev = torch.device("cuda", 0)
    shapes = split_precision_shapes()
    vs = pt.variants()
    ids = [v["id"] for v in vs if v["kind"] != 0 or (v["fma2"] and v["bm"] * v["bn"] >= 4096 and v["splitk"] <= 4)]
    out_dir = args.out_dir or tempfile.mkdtemp(prefix="ptsplit_")
    os.makedirs(out_dir, exist_ok=True)
    table = os.path.join(out_dir, "splitprec_table.csv")
    t0 = time.perf_counter()
    pt.tune(shapes, table, ids=ids, reps_min=3, reps_max=10, target_ms=10.0)
    tune_s = time.perf_counter() - t0
    import csv
    rows = list(csv.DictReader(open(table)))
    res = []
    for (M, N, K) in shapes:
        best = {}
        for r in rows:
            if (int(r["M"]), int(r["N"]), int(r["K"])) != (M, N, K) or not int(r["valid"]):
                continue
            kind = pt.variant(pt.variant_by_name(r["variant"]))["kind"]
            t = float(r["median_ms"])
            if kind not in best or t < best[kind][0]:
                best[kind] = (t, r["variant"])
        entry = {"shape": [M, N, K]}
        for kind, label in KIND_LABELS.items():
            if kind in best:
                t, name = best[kind]
                entry[label] = {"variant": name, "ms": t, "tflops": 2.0 * M * N * K / (t * 1e-3) / 1e12}
        res.append(entry)
    torch.backends.cuda.matmul.allow_tf32 = True
    X = torch.randn(8192, 8192, device=dev)
    Y = torch.randn(8192, 8192, device=dev)
    for _ in range(3):
        torch.matmul(X, Y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        torch.matmul(X, Y)
    e1.record()
    torch.cuda.synchronize()
    tf32 = 10 * 2.0 * 8192 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = False
    print(json.dumps({"mode": "splitprec", "inputs": "sign * 2^U[-10,10], seed 3", "tune_s": tune_s,
                      "tf32_cublas_tflops_8192": tf32, "shapes": res}))
    return 0


def report_noalloc(args):
    """pt_sgemm_3xtf32_noalloc against the registry's tc3xtf32_m128n128_p3
    (the same split and kernel with a library workspace) on 1536^3 and
    1024 x 2048 x 1024, U[-1,1]: mean call time over 50 launches each,
    CUDA events on one stream."""
    import ctypes

    import torch

    import paper_2507_15277_gb300 as pt
    from paper_2507_15277_gb300 import _lib
    from workloads import matrix
    dev = torch.device("cuda", 0)
    lib = _lib.lib()
    stream = torch.cuda.Stream(dev)
    vid = pt.variant_by_name("tc3xtf32_m128n128_p3")
    res = []
    for (M, N, K) in ((1536, 1536, 1536), (1024, 2048, 1024)):
        A = torch.from_numpy(matrix("uniform", 1, M, K)).to(dev)
        B = torch.from_numpy(matrix("uniform", 2, K, N)).to(dev)
        C = torch.empty((M, N), device=dev)

        def noalloc():
            rc = lib.pt_sgemm_3xtf32_noalloc(b"N", b"N", M, N, K, 1.0, ctypes.c_void_p(A.data_ptr()), K,
                                             ctypes.c_void_p(B.data_ptr()), N, 0.0, ctypes.c_void_p(C.data_ptr()),
                                             N, ctypes.c_void_p(stream.cuda_stream))
            if rc:
                raise RuntimeError(lib.pt_last_error())

        def twin():
            pt.sgemm(A, B, C, variant=vid, stream=stream)

        entry = {"shape": [M, N, K]}
        for name, fn in (("noalloc", noalloc), ("tc3xtf32_m128n128_p3", twin)):
            with torch.cuda.stream(stream):
                for _ in range(5):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(50):
                    fn()
                e1.record(stream)
                stream.synchronize()
            ms = e0.elapsed_time(e1) / 50
            entry[name] = {"ms": ms, "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12}
        res.append(entry)
    print(json.dumps({"mode": "noalloc", "shapes": res}))
    return 0


def _normalised(C, R, K, amax, bmax):
    """max |C - R| / (K max|A| max|B|): the normalised error of a result
    against a reference result."""
    import numpy as np
    return float(np.abs(np.asarray(C, np.float64) - np.asarray(R, np.float64)).max() / (K * amax * bmax))


def _ranks(x):
    """Ranks 0..n-1 of x (ties get the mean of their ranks)."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    order = np.argsort(x, kind="mergesort")
    r = np.empty(len(x), dtype=np.float64)
    r[order] = np.arange(len(x), dtype=np.float64)
    for v in np.unique(x):
        idx = np.nonzero(x == v)[0]
        if len(idx) > 1:
            r[idx] = r[idx].mean()
    return r


def spearman(a, b):
    """Spearman rank correlation of two equal-length samples."""
    import numpy as np
    ra, rb = _ranks(a), _ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = float(np.sqrt((ra * ra).sum() * (rb * rb).sum()))
    return float((ra * rb).sum() / den) if den > 0 else 1.0


def report_stability(args):
    """Timing-table stability: the 64-shape sweep is tuned twice; per shape,
    the Spearman rank correlation of the valid variants' median times between
    the two passes, whether the per-shape best variant is the same, and the
    time the second pass's best needs in the first pass relative to the first
    pass's best (1.0 when the best agrees)."""
    import csv

    import numpy as np

    import paper_2507_15277_gb300 as pt
    from workloads import sweep_shapes
    shapes = sweep_shapes()
    out_dir = args.out_dir or tempfile.mkdtemp(prefix="ptstab_")
    os.makedirs(out_dir, exist_ok=True)
    paths = [os.path.join(out_dir, "pass%d.csv" % i) for i in (1, 2)]
    for path in paths:
        pt.tune(shapes, path, reps_min=5, reps_max=args.tune_reps_max, target_ms=args.tune_target_ms)
    tabs = []
    for path in paths:
        t = {}
        for r in csv.DictReader(open(path)):
            if int(r["valid"]):
                t[(int(r["M"]), int(r["N"]), int(r["K"]), r["variant"])] = float(r["median_ms"])
        tabs.append(t)
    per = []
    for (M, N, K) in shapes:
        names = sorted({v for (m, n, k, v) in tabs[0] if (m, n, k) == (M, N, K)} &
                       {v for (m, n, k, v) in tabs[1] if (m, n, k) == (M, N, K)})
        a = [tabs[0][(M, N, K, v)] for v in names]
        b = [tabs[1][(M, N, K, v)] for v in names]
        best1, best2 = names[int(np.argmin(a))], names[int(np.argmin(b))]
        per.append({"shape": [M, N, K], "variants": len(names), "spearman": spearman(a, b),
                    "same_best": best1 == best2, "pass1_time_of_pass2_best_rel": tabs[0][(M, N, K, best2)] / min(a)})
    rho = [p["spearman"] for p in per]
    print(json.dumps({"mode": "stability", "shapes": len(per),
                      "spearman_median": float(np.median(rho)), "spearman_min": float(np.min(rho)),
                      "same_best_fraction": sum(p["same_best"] for p in per) / len(per),
                      "geomean_pass1_time_of_pass2_best_rel":
                          float(np.exp(np.mean(np.log([p["pass1_time_of_pass2_best_rel"] for p in per])))),
                      "per_shape": per}))
    return 0


def cpu_oracle_square():
    """CPU-baseline leg: the FP64 oracle timed at 256^3, 1024^3 and 4096^3,
    on one thread and on all of the host's threads (GFLOP/s), with the host
    CPU model.  The one-thread 4096^3 run is bounded to 256 of the rows."""
    import numpy as np

    from oracle import gemm as og
    from workloads import matrix
    model = ""
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    nmax = og.num_threads()
    res = []
    for n in (256, 1024, 4096):
        A = matrix("uniform", 1, n, n)
        B = matrix("uniform", 2, n, n)
        for threads in (1, nmax):
            og.set_threads(threads)
            rows = None
            if threads == 1 and n == 4096:
                rows = np.arange(256)
            og.gemm(A[:8], B, M=8, N=n, K=n)  # warm
            t0 = time.perf_counter()
            og.gemm(A, B, M=n, N=n, K=n, rows=rows)
            dt = time.perf_counter() - t0
            m = n if rows is None else len(rows)
            res.append({"shape": [n, n, n], "threads": threads, "rows": m, "s": dt,
                        "gflops": 2.0 * m * n * n / dt / 1e9})
    og.set_threads(nmax)
    return {"cpu": model, "threads_max": nmax, "runs": res}


def report_oracle(args):
    """The CPU-baseline leg's square-size timings by themselves."""
    print(json.dumps(dict(mode="oracle", **cpu_oracle_square())))
    return 0


def report_autograd(args):
    """Y = X W with X[4096,1024], W[1024,4096] ~ N(0, 0.02^2), G ~ N(0,1)
    (seed 4): the three products (NN forward, NT dX = G W^T, TN dW = X^T G)
    are tuned over every variant, k = 3 are selected on them, and forward +
    backward through the autograd Function is timed against torch.matmul in
    FP32 (TF32 off); errors of Y, dX, dW on sampled rows against the
    library's compensated-dot reference kernel (the FP64 oracle checks the
    gradients in the tests)."""
    import numpy as np
    import torch

    import paper_2507_15277_gb300 as pt
    from paper_2507_15277_gb300.autograd import matmul
    from workloads import matrix
    dev = torch.device("cuda", 0)
    Mx, Kx, Nw = 4096, 1024, 4096
    X = matrix("normal", 4, Mx, Kx, std=0.02)
    W = matrix("normal", 104, Kx, Nw, std=0.02)
    G = matrix("normal", 204, Mx, Nw)
    shapes = [(Mx, Nw, Kx, "N", "N"), (Mx, Kx, Nw, "N", "T"), (Kx, Nw, Mx, "T", "N")]
    out_dir = args.out_dir or tempfile.mkdtemp(prefix="ptgrad_")
    os.makedirs(out_dir, exist_ok=True)
    table = os.path.join(out_dir, "autograd_table.csv")
    pt.tune(shapes, table, reps_min=3, reps_max=10, target_ms=5.0)
    manifest = os.path.join(out_dir, "autograd_k3.json")
    ids, _ = pt.select(table, [0, 1, 2], 3, manifest=manifest)
    pt.load_manifest(manifest)
    Xd = torch.from_numpy(X).to(dev).requires_grad_(True)
    Wd = torch.from_numpy(W).to(dev).requires_grad_(True)
    Gd = torch.from_numpy(G).to(dev)

    def ours():
        Y = matmul(Xd, Wd)
        Y.backward(Gd)
        return Y

    def ref():
        Y = torch.matmul(Xd, Wd)
        Y.backward(Gd)
        return Y

    torch.backends.cuda.matmul.allow_tf32 = False
    torch.set_float32_matmul_precision("highest")
    res = {}
    for name, fn in (("pt_sgemm", ours), ("torch_fp32", ref)):
        for _ in range(3):
            Xd.grad = None
            Wd.grad = None
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            Xd.grad = None
            Wd.grad = None
            Y = fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        res[name] = {"ms": ms, "tflops": 3 * 2.0 * Mx * Nw * Kx / (ms * 1e-3) / 1e12}
    Xd.grad = None
    Wd.grad = None
    Y = ours()
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    rx = np.sort(rng.choice(Mx, 64, replace=False))
    rw = np.sort(rng.choice(Kx, 64, replace=False))
    with torch.no_grad():
        refs = (pt.reference(Xd.detach(), Wd.detach()), pt.reference(Gd, Wd.detach(), transB="T"),
                pt.reference(Xd.detach(), Gd, transA="T"))
    err = {
        "Y": _normalised(Y.detach()[rx].cpu().numpy(), refs[0][rx].cpu().numpy(), Kx, np.abs(X).max(),
                         np.abs(W).max()),
        "dX": _normalised(Xd.grad[rx].cpu().numpy(), refs[1][rx].cpu().numpy(), Nw, np.abs(G).max(),
                          np.abs(W).max()),
        "dW": _normalised(Wd.grad[rw].cpu().numpy(), refs[2][rw].cpu().numpy(), Mx, np.abs(X).max(),
                          np.abs(G).max()),
    }
    print(json.dumps({"mode": "autograd", "shapes": [list(s[:3]) + [s[3] + s[4]] for s in shapes],
                      "kappa": [pt.variant(i)["name"] for i in ids],
                      "picks": [pt.variant(pt.selected_variant(m, n, k, ta, tb))["name"] for m, n, k, ta, tb in shapes],
                      "timing": res, "errors": err}))
    return 0


def single(args):
    """One variant on one shape, `warmup` + `steps` launches (for ncu captures)."""
    import torch

    import paper_2507_15277_gb300 as pt
    from workloads import matrix
    M, N, K = (int(x) for x in args.single.split(","))
    vid = pt.variant_by_name(args.variant) if args.variant else pt.default_variant()
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(matrix("uniform", 1, M, K)).to(dev)
    B = torch.from_numpy(matrix("uniform", 2, K, N)).to(dev)
    C = torch.empty((M, N), device=dev)
    for _ in range(args.warmup):
        pt.sgemm(A, B, C, variant=vid)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pt.sgemm(A, B, C, variant=vid)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # The main GEMM kernel alone (library events around it; excludes the
    # tensor-core versions' split kernel).
    pt.kernel_timer_start()
    for _ in range(args.steps):
        pt.sgemm(A, B, C, variant=vid)
    kms, n = pt.kernel_timer_stop()
    kms /= max(1, n)
    print(json.dumps({"mode": "single", "variant": pt.variant(vid)["name"], "shape": [M, N, K], "ms": ms,
                      "tflops": 2.0 * M * N * K / (ms * 1e-3) / 1e12, "kernel_ms": kms,
                      "kernel_tflops": 2.0 * M * N * K / (kms * 1e-3) / 1e12}))
    return 0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- replica coordination (host side; the data path has no collective) --------------
def shared_out_dir(out_dir, rank, world):
    """The folder for the timing table and manifests, the same on every rank:
    the given one, else a fresh one that rank 0 creates and broadcasts."""
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        return out_dir
    if world == 1:
        return tempfile.mkdtemp(prefix="ptbench_")
    import torch.distributed as dist
    obj = [tempfile.mkdtemp(prefix="ptbench_") if rank == 0 else None]
    dist.broadcast_object_list(obj, src=0)
    return obj[0]


def share_manifest(pt, manifest_path, rank, world, make):
    """Rank 0 runs make() (tuning + selection, which writes manifest_path);
    after a barrier every rank installs the same manifest."""
    if rank == 0:
        make()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    pt.load_manifest(manifest_path)


def whole_job(times_ms, world, device=None):
    """Max of each time over the ranks (the job ends with its slowest rank)."""
    import torch
    t = torch.tensor(times_ms, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


# ---- clocks ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_id

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    """Measured peaks of this GPU pool (MEASURED_PEAKS.json), if present."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def source_sha256(files):
    """sha256 over the named kernel sources (csrc/), in the given order."""
    import hashlib
    src = os.path.join(ROOT, "paper_2507_15277_gb300", "csrc")
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(src, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_for(kernel, shape):
    """DRAM bytes per launch of the main GEMM kernel from the committed ncu
    summary of this kernel and shape (profiles/traffic.json), or None when no
    capture of the current kernel source exists (each entry names the source
    files its kernel is built from and their sha256 at capture time)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    for e in rec.get("captures", []):
        if e.get("kernel") == kernel and tuple(e.get("shape", ())) == tuple(shape):
            try:
                if e.get("source_sha256") == source_sha256(e.get("source_files", [])):
                    return e.get("dram_bytes")
            except OSError:
                return None
    return None


# ---- CPU oracle baseline -----------------------------------------------------------------
def per_shape_times(calls, stream, reps=3):
    """Median device time of each call in `calls` (issued in order on `stream`).

    The calls are captured once in a CUDA graph with a timing event recorded
    between consecutive calls, and the graph is replayed `reps` times, so host
    launch latency never sits between two events.  The event nodes also
    separate the calls, so no call overlaps its neighbour.  Where a timing
    event cannot be captured, the calls are issued eagerly between events
    instead.  Returns (per-call ms, method)."""
    import torch

    n = len(calls)
    times = [[] for _ in range(n)]
    try:
        ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(n + 1)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(g, stream=stream):
                ev[0].record(stream)
                for i, c in enumerate(calls):
                    c()
                    ev[i + 1].record(stream)
        torch.cuda.synchronize()
        for _ in range(reps):
            g.replay()
            torch.cuda.synchronize()
            for i in range(n):
                times[i].append(ev[i].elapsed_time(ev[i + 1]))
        del g
        method = "graph replay, timing events between calls"
    except (RuntimeError, TypeError):
        torch.cuda.synchronize()
        times = [[] for _ in range(n)]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        with torch.cuda.stream(stream):
            for _ in range(reps):
                ev[0].record(stream)
                for i, c in enumerate(calls):
                    c()
                    ev[i + 1].record(stream)
                stream.synchronize()
                for i in range(n):
                    times[i].append(ev[i].elapsed_time(ev[i + 1]))
        method = "eager, timing events between calls (includes host launch gaps)"
    return [statistics.median(x) for x in times], method


def per_shape_stream_times(calls, stream, repeat=10):
    """Device time of each call when it runs back to back with itself:
    `repeat` launches of the call between two timing events, all shapes in
    one captured graph replayed once (after one warm replay).  Launch
    overlap is then as in the timed step, but the shape's inputs are in L2
    after its first launch.  Returns per-call ms (total / repeat)."""
    import torch
    n = len(calls)
    ev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(n + 1)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            ev[0].record(stream)
            for i, c in enumerate(calls):
                for _ in range(repeat):
                    c()
                ev[i + 1].record(stream)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
    out = [ev[i].elapsed_time(ev[i + 1]) / repeat for i in range(n)]
    del g
    return out


def cpu_oracle_sample(shapes, rows_per_shape, seed_base=1000):
    """Times the FP64 CPU oracle on the first `rows_per_shape` rows of every
    shape (all rows when M is smaller).  Returns (TFLOP/s, seconds, cores, flops)."""
    from oracle import gemm as og
    from workloads import matrix
    og.gemm(matrix("uniform", 0, 8, 8), matrix("uniform", 1, 8, 8))  # load / build the oracle
    work = []
    for i, (M, N, K) in enumerate(shapes):
        r = min(M, rows_per_shape)
        A = matrix("uniform", seed_base + i, r, K)  # the first r rows of A (same values)
        B = matrix("uniform", 100000 + seed_base + i, K, N)
        work.append((A, B, r, N, K))
    flops = 0.0
    t0 = time.perf_counter()
    for A, B, r, N, K in work:
        og.gemm(A, B)
        flops += 2.0 * r * N * K
    dt = time.perf_counter() - t0
    return flops / dt / 1e12, dt, og.num_threads(), flops


KIND_LABELS = {0: "fp32_simt", 1: "3xtf32", 2: "bf16x3", 3: "3xf16"}
# Tensor-core kinds: (MMA products per FP32 product, MMA input type, its
# dense rate relative to BF16).
TC_KINDS = {1: (3, "tf32", 1.1 / 2.25), 2: (6, "bf16", 1.0), 3: (3, "f16", 1.0)}


def selection_by_kind(pt, table, train, held, out_dir):
    """PortabilityTune (Eq. 1) run on one kind's variants at a time: the
    table restricted to FP32 SIMT, 3xTF32 or BF16x3 rows.  For k = 1, 2, 4, 8
    the held-out geomean of t_best / t(best member) is scored against that
    kind's own per-shape best and against the per-shape best of the whole
    family (every kind meets the same 2e-6 error bound)."""
    import csv
    with open(table) as f:
        rows = list(csv.DictReader(f))
    fields = list(rows[0].keys()) if rows else []
    kind_of = {}
    out = {}
    for kind, label in KIND_LABELS.items():
        sub = []
        for r in rows:
            if r["variant"] not in kind_of:
                kind_of[r["variant"]] = pt.variant(pt.variant_by_name(r["variant"]))["kind"]
            if kind_of[r["variant"]] == kind:
                sub.append(r)
        if not sub:
            continue
        path = os.path.join(out_dir, "table_%s.csv" % label)
        with open(path, "w", newline="") as f:
            w = csv.DictWriter(f, fieldnames=fields)
            w.writeheader()
            w.writerows(sub)
        res = {"variants": len({r["variant"] for r in sub})}
        for k in (1, 2, 4, 8):
            ids, _ = pt.select(path, train, k)
            res["k%d" % k] = {"own_best_pct": round(100 * pt.score(path, held, ids), 2),
                              "family_best_pct": round(100 * pt.score(table, held, ids), 2)}
        out[label] = res
    return out


def best_simt_from_table(pt, table, shape=(4096, 4096, 4096)):
    """Fastest FP32 SIMT variant of the timing table on one shape (median)."""
    import csv
    best = None
    with open(table) as f:
        for r in csv.DictReader(f):
            if (int(r["M"]), int(r["N"]), int(r["K"])) != shape or not int(r["valid"]):
                continue
            if pt.variant(pt.variant_by_name(r["variant"]))["kind"] != 0:
                continue
            if best is None or float(r["median_ms"]) < best[1]:
                best = (r["variant"], float(r["median_ms"]))
    return best


def config1_timing(pt, dev, stream, reps=200):
    """The fixed single-GEMM workload: 256^3, NN, alpha = 1, beta = 0, U[-1,1]
    (seeds 1 and 2), the 128x128x8 cp.async variant; mean of `reps` launches
    replayed from a CUDA graph, CUDA events."""
    import torch
    from workloads import matrix
    name = "s128x128x8_w32x64_t8x8_kl1_v4_p2_sk1_cpm"
    vid = pt.variant_by_name(name)
    A = torch.from_numpy(matrix("uniform", 1, 256, 256)).to(dev)
    B = torch.from_numpy(matrix("uniform", 2, 256, 256)).to(dev)
    C = torch.empty((256, 256), device=dev)
    with torch.cuda.stream(stream):
        pt.sgemm(A, B, C, variant=vid, stream=stream)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(reps):
                pt.sgemm(A, B, C, variant=vid, stream=stream)
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return name, ms


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from workloads import sweep_shapes
    shapes = sweep_shapes()
    rows = max(1, args.cpu_rows // 4)
    for _ in range(args.warmup):
        cpu_oracle_sample(shapes[:4], 8)
    vals, secs, flops_total = [], 0.0, 0.0
    cores = 1
    for _ in range(args.steps):
        v, dt, cores, fl = cpu_oracle_sample(shapes, rows)
        vals.append(v)
        secs += dt
        flops_total += fl
    value = flops_total / secs / 1e12
    sample = "FP64 CPU oracle (i-k-j triple loop, OpenMP) on the first %d rows of each of the 64 sweep shapes per step" % rows
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---- our arm ----------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.single:
        return single(args)
    if args.report == "splitprec":
        return report_splitprec(args)
    if args.report == "grouped":
        return report_grouped(args)
    if args.report == "stability":
        return report_stability(args)
    if args.report == "oracle":
        return report_oracle(args)
    if args.report == "autograd":
        return report_autograd(args)
    if args.report == "noalloc":
        return report_noalloc(args)

    import numpy as np
    import torch

    import paper_2507_15277_gb300 as pt
    from workloads import matrix, parity_split, random_split, sweep_shapes

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    shapes = sweep_shapes()
    train, held = parity_split()
    out_dir = shared_out_dir(args.out_dir, rank, world)
    table = args.table or os.path.join(out_dir, "table.csv")
    info = {}

    # ---- data collection + selection (rank 0; other ranks reuse its manifest) ----
    def collect_and_select():
        t0 = time.perf_counter()
        if not args.table:
            pt.tune(shapes, table, reps_min=5, reps_max=args.tune_reps_max, target_ms=args.tune_target_ms)
        info["tune_s"] = time.perf_counter() - t0
        sel = {}
        t0 = time.perf_counter()
        for k in range(1, 9):
            man = os.path.join(out_dir, "kappa_k%d.json" % k)
            ids, g_train = pt.select(table, train, k, manifest=man)
            sel[k] = {
                "ids": ids,
                "names": [pt.variant(i)["name"] for i in ids],
                "train": g_train,
                "heldout_best_of_set": pt.score(table, held, ids),
                "heldout_selector": pt.score(table, held, mode=pt.PT_SCORE_SELECTOR, manifest=man),
            }
        info["select_s"] = time.perf_counter() - t0
        # Mean and spread over 10 seeded random 32/32 splits.
        rs = {}
        for k in (1, 2, 4, 8):
            vals = []
            for seed in range(10):
                tr, he = random_split(seed)
                ids, _ = pt.select(table, tr, k)
                vals.append(pt.score(table, he, ids))
            rs[k] = (statistics.mean(vals), statistics.pstdev(vals))
        info["random_splits"] = rs
        info["selection"] = sel
        # The paper's alternative implementations (Section IV-C) on the same
        # split: held-out best-of-set and selector-realised scores and the
        # time each selection takes.
        comp = {}
        for mname, method in (("portabilitytune", pt.PT_SELECT_AUTO), ("kmeans", pt.PT_SELECT_KMEANS),
                              ("tree", pt.PT_SELECT_TREE)):
            comp[mname] = {}
            for k in (1, 2, 4, 8):
                man = os.path.join(out_dir, "sel_%s_k%d.json" % (mname, k))
                t0 = time.perf_counter()
                ids, g_train = pt.select(table, train, k, method=method, manifest=man)
                dt = time.perf_counter() - t0
                comp[mname]["k%d" % k] = {
                    "n_ids": len(ids), "train_pct": 100 * g_train,
                    "heldout_pct": 100 * pt.score(table, held, ids),
                    "heldout_selector_pct": 100 * pt.score(table, held, mode=pt.PT_SCORE_SELECTOR, manifest=man),
                    "select_s": dt}
        info["selectors"] = comp
        info["by_kind"] = selection_by_kind(pt, table, train, held, out_dir)
    manifest = os.path.join(out_dir, "kappa_k%d.json" % args.k)
    share_manifest(pt, manifest, rank, world, collect_and_select)

    # ---- inputs: pinned host copies and resident device buffers ----
    # All shapes' A and B (shape order, A then B) live in one pinned host
    # buffer and one device buffer, and all C in another pair, so that the
    # end-to-end pipeline moves a group of consecutive shapes with one copy
    # per direction.  Every view starts at a multiple of 128 x 128 floats.
    in_off, out_off, o_in, o_out = [], [], 0, 0
    for (M, N, K) in shapes:
        in_off.append(o_in)
        out_off.append(o_out)
        o_in += M * K + K * N
        o_out += M * N
    in_off.append(o_in)
    out_off.append(o_out)
    host_in = torch.empty(o_in, dtype=torch.float32, pin_memory=True)
    host_out = torch.empty(o_out, dtype=torch.float32, pin_memory=True)
    dev_in = torch.empty(o_in, dtype=torch.float32, device=dev)
    dev_out = torch.empty(o_out, dtype=torch.float32, device=dev)
    hostA, hostB, hostC, devA, devB, devC = [], [], [], [], [], []
    flops = []
    for i, (M, N, K) in enumerate(shapes):
        o = in_off[i]
        hostA.append(host_in[o:o + M * K].view(M, K))
        hostB.append(host_in[o + M * K:o + M * K + K * N].view(K, N))
        hostC.append(host_out[out_off[i]:out_off[i] + M * N].view(M, N))
        devA.append(dev_in[o:o + M * K].view(M, K))
        devB.append(dev_in[o + M * K:o + M * K + K * N].view(K, N))
        devC.append(dev_out[out_off[i]:out_off[i] + M * N].view(M, N))
        hostA[i].copy_(torch.from_numpy(matrix("uniform", 1000 + i, M, K)))
        hostB[i].copy_(torch.from_numpy(matrix("uniform", 100000 + 1000 + i, K, N)))
        flops.append(2.0 * M * N * K)
    dev_in.copy_(host_in)
    dev_out.zero_()
    torch.cuda.synchronize()
    step_flops = sum(flops)
    picks = [pt.selected_variant(M, N, K, A=devA[i], B=devB[i], C=devC[i]) for i, (M, N, K) in enumerate(shapes)]
    stream = torch.cuda.Stream(dev)

    def step():
        for i in range(len(shapes)):
            pt.sgemm(devA[i], devB[i], devC[i], stream=stream)

    # Capture the step once as a CUDA graph (64 launches, no host work).
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        step()  # warm (attribute setup, descriptors)
        stream.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            step()
    torch.cuda.synchronize()

    # ---- per-shape times: timing events between the calls of a captured graph ----
    shape_ms, per_shape_timing = per_shape_times(
        [lambda i=i: pt.sgemm(devA[i], devB[i], devC[i], stream=stream) for i in range(len(shapes))], stream)

    try:
        shape_ms_stream = per_shape_stream_times(
            [lambda i=i: pt.sgemm(devA[i], devB[i], devC[i], stream=stream) for i in range(len(shapes))], stream)
    except (RuntimeError, TypeError):
        shape_ms_stream = [None] * len(shapes)

    # ---- timed region: graph replays ----
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    clk = clocks.stop()

    # Eager (no graph) steps: the same launches issued from Python each step.
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            step()
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1)

    # ---- end to end: host inputs in, host result out, every step ----
    # A three-stage pipeline over groups of consecutive shapes (about equal
    # bytes per group), one stream per stage: the host-to-device copy of group
    # g+1 runs while group g computes and the results of group g-1 are copied
    # back (events order the stages of a group).  One copy per group and
    # direction keeps the per-copy overhead of the small shapes off the link.
    # Consecutive steps use two sets of device buffers in turn, so a step's
    # copies need not wait for the previous step's GEMMs and copies of the
    # same group: both copy directions stream without gaps.  This is how a
    # user of the API overlaps host data with compute; the host link, not the
    # GEMMs, bounds it.
    h2d = sum(a.numel() * 4 + b.numel() * 4 for a, b in zip(hostA, hostB))
    d2h = sum(c.numel() * 4 for c in hostC)
    n_groups = 16
    target = (in_off[-1] + out_off[-1]) / n_groups
    groups, lo, acc = [], 0, 0.0
    for i in range(len(shapes)):
        acc += (in_off[i + 1] - in_off[i]) + (out_off[i + 1] - out_off[i])
        if acc >= target or i == len(shapes) - 1:
            groups.append((lo, i + 1))
            lo, acc = i + 1, 0.0
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    # the second set of device buffers (the first is the resident one)
    dev_in2 = torch.empty(o_in, dtype=torch.float32, device=dev)
    dev_out2 = torch.empty(o_out, dtype=torch.float32, device=dev)
    dev_in2.copy_(dev_in)
    bufs = [(dev_in, dev_out, devA, devB, devC),
            (dev_in2, dev_out2,
             [dev_in2[in_off[i]:in_off[i] + M * K].view(M, K) for i, (M, N, K) in enumerate(shapes)],
             [dev_in2[in_off[i] + M * K:in_off[i + 1]].view(K, N) for i, (M, N, K) in enumerate(shapes)],
             [dev_out2[out_off[i]:out_off[i + 1]].view(M, N) for i, (M, N, K) in enumerate(shapes)])]
    ev_in = [[torch.cuda.Event() for _ in groups] for _ in bufs]
    ev_done = [[torch.cuda.Event() for _ in groups] for _ in bufs]
    ev_out = [[torch.cuda.Event() for _ in groups] for _ in bufs]

    def e2e_step(p):
        d_in, d_out, dA, dB, dC = bufs[p]
        for g, (a, b) in enumerate(groups):
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_done[p][g])  # the GEMMs of group g that last used this buffer set are done
                d_in[in_off[a]:in_off[b]].copy_(host_in[in_off[a]:in_off[b]], non_blocking=True)
                ev_in[p][g].record(s_in)
            stream.wait_event(ev_in[p][g])
            stream.wait_event(ev_out[p][g])  # the last copy of group g's results out of this set has finished
            for i in range(a, b):
                pt.sgemm(dA[i], dB[i], dC[i], stream=stream)
            ev_done[p][g].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[p][g])
                host_out[out_off[a]:out_off[b]].copy_(d_out[out_off[a]:out_off[b]], non_blocking=True)
                ev_out[p][g].record(s_out)

    for p in range(len(bufs)):
        for g in range(len(groups)):
            ev_done[p][g].record(stream)
            ev_out[p][g].record(s_out)
    for w in range(2):
        e2e_step(w % 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    s_in.wait_stream(stream)
    for st in range(args.steps):
        e2e_step(st % 2)
    stream.wait_stream(s_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_wall = time.perf_counter() - t0
    e2e_ms = e0.elapsed_time(e1)

    # Overlap of the three stages in one more (untimed) pipelined step: timing
    # events around every copy and GEMM group give each stage's busy time;
    # with full overlap the step takes about the longest stage, without any
    # it takes their sum.
    ev_t = {}

    def timed_e2e_step():
        for g, (a, b) in enumerate(groups):
            ts = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            ev_t[g] = ts
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_done[0][g])
                ts[0].record(s_in)
                dev_in[in_off[a]:in_off[b]].copy_(host_in[in_off[a]:in_off[b]], non_blocking=True)
                ts[1].record(s_in)
                ev_in[0][g].record(s_in)
            stream.wait_event(ev_in[0][g])
            stream.wait_event(ev_out[0][g])
            ts[2].record(stream)
            for i in range(a, b):
                pt.sgemm(devA[i], devB[i], devC[i], stream=stream)
            ts[3].record(stream)
            ev_done[0][g].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[0][g])
                ts[4].record(s_out)
                host_out[out_off[a]:out_off[b]].copy_(dev_out[out_off[a]:out_off[b]], non_blocking=True)
                ts[5].record(s_out)
                ev_out[0][g].record(s_out)

    torch.cuda.synchronize()
    t_first = torch.cuda.Event(enable_timing=True)
    t_first.record(stream)
    s_in.wait_stream(stream)
    timed_e2e_step()
    stream.wait_stream(s_out)
    t_last = torch.cuda.Event(enable_timing=True)
    t_last.record(stream)
    torch.cuda.synchronize()
    busy = [sum(ev_t[g][2 * st].elapsed_time(ev_t[g][2 * st + 1]) for g in ev_t) for st in range(3)]
    overlap = {"step_ms": t_first.elapsed_time(t_last), "h2d_busy_ms": busy[0], "gemm_busy_ms": busy[1],
               "d2h_busy_ms": busy[2]}
    overlap["overlap_factor"] = sum(busy) / overlap["step_ms"]

    # Copy-engine rates alone (context for e2e): one step's input and output
    # copies, each direction by itself.
    def copies_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(reps):
                fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    h2d_ms = copies_ms(lambda: [dev_in[in_off[a]:in_off[b]].copy_(host_in[in_off[a]:in_off[b]], non_blocking=True)
                                for a, b in groups])
    d2h_ms = copies_ms(lambda: [host_out[out_off[a]:out_off[b]].copy_(dev_out[out_off[a]:out_off[b]],
                                                                      non_blocking=True) for a, b in groups])

    # Whole-job numbers: max time over ranks, units over all ranks.
    elapsed_ms, e2e_ms, eager_ms = whole_job([elapsed_ms, e2e_ms, eager_ms], world, dev)
    value = world * step_flops * args.steps / (elapsed_ms * 1e-3) / 1e12
    e2e_value = world * step_flops * args.steps / (e2e_ms * 1e-3) / 1e12

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel (largest share of the step) ----
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    dom = max(range(len(shapes)), key=lambda i: shape_ms[i])
    M, N, K = shapes[dom]
    dom_ms = shape_ms[dom]
    f_max = 2070.0
    fp32_peak = sms * 128 * 2 * f_max * 1e6 / 1e12
    f_med = clk.get("sm_mhz")
    peaks = measured_peaks()
    dvar = pt.variant(picks[dom])
    # The dominant kernel's own launches: CUDA events recorded by the library
    # directly around its main GEMM kernel (for the tensor-core versions this
    # excludes the split kernel, reported separately as split_ms).
    call_ms = dom_ms
    reps = 20
    with torch.cuda.stream(stream):
        for _ in range(3):
            pt.sgemm(devA[dom], devB[dom], devC[dom], stream=stream)
        stream.synchronize()
        pt.kernel_timer_start()
        e0.record(stream)
        for _ in range(reps):
            pt.sgemm(devA[dom], devB[dom], devC[dom], stream=stream)
        e1.record(stream)
        total_ms, n_timed = pt.kernel_timer_stop()
    stream.synchronize()
    call_ms = e0.elapsed_time(e1) / reps
    dom_ms = total_ms / max(1, n_timed)
    if dvar["kind"] == 0:
        # FP32 FMA on the CUDA cores: 2MNK flops against the FP32 ALU peak.
        achieved = flops[dom] / (dom_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "peak_basis": "FP32 FMA: %d SMs x 128 lanes x 2 flop x %.0f MHz (max SM clock)" % (sms, f_max),
                    "frac_at_sampled_clock": (achieved / (sms * 256 * f_med * 1e6 / 1e12)) if f_med else None}
    else:
        # Split-precision tensor-core kernel: the tensor pipe executes
        # (products per FP32 product) x 2MNK flops of TF32 or BF16 MMAs.
        nprod, dt, ratio = TC_KINDS[dvar["kind"]]
        achieved = nprod * flops[dom] / (dom_ms * 1e-3) / 1e12
        bf16 = peaks.get("bf16_tflops") or 1900.0
        bf16_sus = peaks.get("bf16_tflops_sustained") or 1700.0
        roofline = {"bound": "tensor", "achieved": achieved, "peak": bf16 * ratio, "unit": "TFLOP/s",
                    "peak_basis": "%s dense tensor peak = measured cuBLAS bf16 burst %.1f TFLOP/s (of measured) x "
                                  "nominal %s/bf16 ratio %.3f; achieved counts %d MMA products per FP32 product"
                                  % (dt, bf16, dt, ratio, nprod),
                    "frac_vs_sustained": achieved / (bf16_sus * ratio),
                    "fp32_equivalent_tflops": flops[dom] / (dom_ms * 1e-3) / 1e12,
                    "fp32_equivalent_frac_of_fp32_peak": flops[dom] / (dom_ms * 1e-3) / 1e12 / fp32_peak}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    # The whole call (split kernel + GEMM kernel for the tensor-core versions).
    roofline["call_frac"] = roofline["achieved"] * dom_ms / call_ms / roofline["peak"]
    roofline.update({"traffic": traffic_for(dvar["name"], (M, N, K)), "kernel": dvar["name"], "shape": [M, N, K],
                     "kernel_ms": dom_ms, "launches_timed": n_timed, "call_ms": call_ms,
                     "split_ms": (call_ms - dom_ms) if dvar["kind"] != 0 else 0.0,
                     "share_of_step": shape_ms[max(range(len(shapes)), key=lambda i: shape_ms[i])] / sum(shape_ms)})
    peak = fp32_peak

    # cuBLAS SGEMM (FP32, TF32 off) on the same shapes, as context.
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.set_float32_matmul_precision("highest")
    with torch.cuda.stream(stream):
        for i in range(len(shapes)):
            torch.matmul(devA[i], devB[i], out=devC[i])
        stream.synchronize()
    cub_ms, _ = per_shape_times(
        [lambda i=i: torch.matmul(devA[i], devB[i], out=devC[i]) for i in range(len(shapes))], stream)
    cublas_tflops = step_flops / (sum(cub_ms) * 1e-3) / 1e12

    c1_name, c1_ms = config1_timing(pt, dev, stream)
    bf16_peak = peaks.get("bf16_tflops") or 1900.0

    def fracs(p, tf):
        kind = pt.variant(p)["kind"]
        d = {"frac_fp32_peak": round(tf / fp32_peak, 4)}
        if kind:
            nprod, _, ratio = TC_KINDS[kind]
            d["frac_tensor_peak"] = round(nprod * tf / (bf16_peak * ratio), 4)
        return d

    best_simt = best_simt_from_table(pt, table)
    small = [i for i in range(len(shapes)) if flops[i] <= 1.1e9]

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, cores, fl = cpu_oracle_sample(shapes, args.cpu_rows)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 CPU oracle on the first %d rows of each of the 64 shapes (%.1f GFLOP, %.1f s)"
                         % (args.cpu_rows, fl / 1e9, dt),
               "square": cpu_oracle_square()}

    sel = info.get("selection", {})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "shapes": 64, "k_deployed": args.k, "variants": pt.num_variants(),
                   "train_split": "parity (i_m+i_n+i_k even) 32/32",
                   "l2": "inputs 1.6 GB (> 129 MB L2) read once per step; no flush needed",
                   "timed": "CUDA graph of the 64 pt_sgemm launches, replayed per step",
                   "compute": "FP32 in/out; per shape the selector picks FP32-FMA SIMT or 3xF16/BF16x3/3xTF32 tensor-core "
                              "splits with FP32 accumulation",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "clocks": clk,
        # per call: SIMT or both operands split in the GEMM kernel: one kernel;
        # otherwise the split kernel and the GEMM kernel
        "gpu_launches": args.steps * sum(1 if pt.variant(p)["kind"] == 0 or "_fab" in pt.variant(p)["name"] else 2
                                         for p in picks),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "wall_s": e2e_wall, "ms_per_step": e2e_ms / args.steps,
                "h2d_gbs_alone": h2d / (h2d_ms * 1e-3) / 1e9, "d2h_gbs_alone": d2h / (d2h_ms * 1e-3) / 1e9,
                "overlap": overlap,
                "pipeline": "3 streams over %d groups of consecutive shapes (about equal bytes), one copy per group "
                            "and direction: H2D of group g+1 | GEMMs of group g | D2H of group g-1; two device "
                            "buffer sets, alternate steps" % len(groups)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "eager_value": world * step_flops * args.steps / (eager_ms * 1e-3) / 1e12,
        "geomean_pct_of_best_heldout": {("k%d" % k): 100 * s["heldout_best_of_set"] for k, s in sel.items()},
        "geomean_pct_of_best_heldout_selector": {("k%d" % k): 100 * s["heldout_selector"] for k, s in sel.items()},
        "geomean_pct_of_best_train": {("k%d" % k): 100 * s["train"] for k, s in sel.items()},
        "random_splits_heldout_pct": {("k%d" % k): [100 * m, 100 * sd] for k, (m, sd) in
                                      info.get("random_splits", {}).items()},
        "kappa": sel.get(args.k, {}).get("names"),
        "selectors": info.get("selectors"),
        "tuning": {"tune_s": info.get("tune_s"), "select_s": info.get("select_s"), "table": table},
        "per_shape": [dict({"shape": list(s), "ms": round(ms, 5), "ms_stream": None if msb is None else round(msb, 5),
                            "tflops": round(f / (ms * 1e-3) / 1e12, 3),
                            "gbs": round(4.0 * (s[0] * s[2] + s[2] * s[1] + s[0] * s[1]) / (ms * 1e-3) / 1e9, 1),
                            "variant": pt.variant(p)["name"], "cublas_tflops": round(f / (cm * 1e-3) / 1e12, 3)},
                           **fracs(p, f / (ms * 1e-3) / 1e12))
                      for s, ms, msb, f, p, cm in zip(shapes, shape_ms, shape_ms_stream, flops, picks, cub_ms)],
        "small_shapes": {"count": len(small), "max_gflop": 1.1, "sum_ms": sum(shape_ms[i] for i in small),
                         "sum_ms_all": sum(shape_ms),
                         "sum_ms_stream": (sum(shape_ms_stream[i] for i in small)
                                           if shape_ms_stream[0] is not None else None)},
        "config1": {"workload": "256^3 NN, alpha=1, beta=0, U[-1,1], fixed 128x128x8 variant", "variant": c1_name,
                    "ms": c1_ms, "tflops": 2.0 * 256 ** 3 / (c1_ms * 1e-3) / 1e12,
                    "frac_fp32_peak": 2.0 * 256 ** 3 / (c1_ms * 1e-3) / 1e12 / fp32_peak},
        "best_fp32_simt_4096": None if best_simt is None else {
            "variant": best_simt[0], "ms": best_simt[1], "tflops": 2.0 * 4096 ** 3 / (best_simt[1] * 1e-3) / 1e12,
            "frac_fp32_peak": 2.0 * 4096 ** 3 / (best_simt[1] * 1e-3) / 1e12 / fp32_peak},
        "selection_by_kind": info.get("by_kind"),
        "context": {"per_shape_timing": per_shape_timing, "cublas_sgemm_tflops": cublas_tflops, "cublas_math": "FP32 (allow_tf32=False, precision highest)",
                    "per_shape_wins_vs_cublas": sum(1 for m, c in zip(shape_ms, cub_ms) if m <= c),
                    "sum_ms_ours": sum(shape_ms), "sum_ms_cublas": sum(cub_ms),
                    "fp32_peak_tflops_at_max_clock": peak, "sms": sms},
    }
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
