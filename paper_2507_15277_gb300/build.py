"""Builds libptsgemm.so in-tree: generates the variant translation units and
compiles everything with nvcc for sm_103a, in parallel.

    python -m paper_2507_15277_gb300.build          # incremental
    python -m paper_2507_15277_gb300.build --force  # from scratch

Objects go to ``_build/`` and the library to ``lib/`` inside the package
(both git-ignored).  The CUDA runtime is linked statically, so the library
loads without PyTorch.
"""

from __future__ import annotations

import glob
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
GEN = os.path.join(BUILD, "gen")
OBJ = os.path.join(BUILD, "obj")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libptsgemm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-Xptxas", "-warn-spills", "-I" + INCLUDE, "-I" + CSRC, "-I" + GEN] + ARCH


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _gen_module():
    sys.path.insert(0, CSRC)
    try:
        import gen_variants
    finally:
        sys.path.pop(0)
    return gen_variants


def _sources():
    _gen_module().generate(GEN)
    cu = sorted(glob.glob(os.path.join(GEN, "variants_*.cu")))
    cu += [os.path.join(CSRC, f) for f in ("registry.cu", "api.cu", "tuner.cu", "tc.cu", "noalloc.cu", "grouped.cu", "grouped_tc.cu")]
    cpp = [os.path.join(CSRC, "select.cpp")]
    return cu, cpp


def _headers():
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hs += glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.join(GEN, "variant_table.inc")]
    return hs


def _stale(obj, src, hdr_mtime):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < hdr_mtime


def _compile(args):
    src, obj = args
    cmd = [nvcc()] + NVCC_FLAGS + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return src, r.stdout + r.stderr
    spills = [ln for ln in (r.stdout + r.stderr).splitlines() if "spill" in ln.lower()]
    with open(obj + ".spills", "w") as f:
        f.write("\n".join(spills))
    os.replace(obj + ".tmp", obj)
    return src, ("\n".join(spills) if spills else None)


_SIMT_ARGS = re.compile(r"SimtI((?:Li-?\d+E){14})E")


def _spilled_variants(objs, fam):
    """Names of variants whose kernels ptxas reported as spilling."""
    by_params = {_gen_module().params_of(v): v["name"] for v in fam}
    drop = set()
    for obj in objs:
        path = obj + ".spills"
        if not os.path.exists(path):
            continue
        for m in _SIMT_ARGS.finditer(open(path).read()):
            params = tuple(int(x) for x in re.findall(r"Li(-?\d+)E", m.group(1)))
            if params in by_params:
                drop.add(by_params[params])
    return drop


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    if force and os.path.isdir(BUILD):
        shutil.rmtree(BUILD)
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cu, cpp = _sources()
    hdr_mtime = max(os.path.getmtime(h) for h in _headers() if os.path.exists(h))
    todo = []
    objs = []
    for src in cu + cpp:
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, src, hdr_mtime):
            todo.append((src, obj))
    jobs = jobs or max(1, os.cpu_count() or 1)
    errors = []
    if todo:
        # Longest first: the generated variant units dominate.
        todo.sort(key=lambda t: 0 if "variants_" in t[0] else 1)
        with ThreadPoolExecutor(max_workers=jobs) as ex:
            for src, msg in ex.map(_compile, todo):
                if msg and ("error" in msg.lower()):
                    errors.append("%s:\n%s" % (src, msg))
                elif msg and verbose:
                    print("%s: %s" % (os.path.basename(src), msg))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n\n".join(errors))
    # Register spills drop a variant from the registry (static pruning rule).
    gm = _gen_module()
    fam, _ = gm.build_family()
    drop = _spilled_variants([o for o in objs if "variants_" in o], fam)
    if fam[0]["name"] in drop:
        raise RuntimeError("the default variant spills registers")
    reg_inc = os.path.join(GEN, "registry_table.inc")
    before = open(reg_inc).read() if os.path.exists(reg_inc) else None
    gm.write_registry(GEN, fam, drop)
    reg_obj = os.path.join(OBJ, "registry.cu.o")
    if open(reg_inc).read() != before or _stale(reg_obj, os.path.join(CSRC, "registry.cu"), os.path.getmtime(reg_inc)):
        src, msg = _compile((os.path.join(CSRC, "registry.cu"), reg_obj))
        if msg and "error" in msg.lower():
            raise RuntimeError("nvcc failed:\n" + msg)
        todo.append((src, reg_obj))
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
