"""Multi-process host logic of bench.py's replica mode (no GPU): two gloo
ranks share one output folder, rank 0 alone selects and writes the manifest
that every rank then installs, and the whole-job time is the maximum over
ranks.  The data path of the replicas has no collective."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pt = pytest.importorskip("paper_2507_15277_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_CSV = ("shape_idx,M,N,K,transA,transB,variant,status,valid,median_ms,mean_ms,min_ms,reps,tflops,gbs,"
              "max_err")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _write_table(path, times, shapes):
    V, S = times.shape
    names = [pt.variant(i)["name"] for i in range(V)]
    with open(path, "w") as f:
        f.write(HEADER_CSV + "\n")
        for s in range(S):
            m, n, k = shapes[s]
            for v in range(V):
                t = times[v, s]
                f.write("%d,%d,%d,%d,N,N,%s,0,1,%.17g,%.17g,%.17g,5,1,1,0\n" % (s, m, n, k, names[v], t, t, t))


def _worker(rank, world, port, table, result_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import paper_2507_15277_gb300 as ptl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = bench.shared_out_dir(None, rank, world)
        dirs = [None] * world
        dist.all_gather_object(dirs, out)
        manifest = os.path.join(out, "kappa.json")
        made = []

        def make():
            made.append(rank)
            ptl.select(table, [0, 1, 2, 3], 2, manifest=manifest)

        bench.share_manifest(ptl, manifest, rank, world, make)
        picks = [ptl.selected_variant(128 * (s + 1), 256, 512) for s in range(6)]
        times = bench.whole_job([1.0 + rank, 5.0 - rank], world)
        with open(os.path.join(result_dir, "r%d.txt" % rank), "w") as f:
            f.write(repr((dirs, made, picks, times)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_share_folder_manifest_and_max_time(tmp_path):
    rng = np.random.default_rng(3)
    shapes = [(128 * (s + 1), 256, 512) for s in range(6)]
    times = np.exp(rng.normal(0, 0.5, size=(6, len(shapes))))
    table = str(tmp_path / "t.csv")
    _write_table(table, times, shapes)
    port = _free_port()
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(2, port, table, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [eval(open(tmp_path / ("r%d.txt" % i)).read()) for i in range(2)]
    dirs0, made0, picks0, times0 = r[0]
    dirs1, made1, picks1, times1 = r[1]
    assert dirs0 == dirs1 and dirs0[0] == dirs0[1]          # one folder for every rank
    assert made0 == [0] and made1 == []                     # only rank 0 tunes and selects
    assert picks0 == picks1                                 # both run the same manifest
    assert times0 == times1 == [2.0, 5.0]                   # max over ranks
