"""Compiles ``gemm_ref.c`` into ``_gemm_ref.so`` next to it (test infrastructure).

Plain gcc; OpenMP when the compiler supports it, single-threaded otherwise.
``-ffp-contract=off`` keeps the FP64 arithmetic identical on x86-64 and
aarch64 hosts.
"""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gemm_ref.c")
LIB = os.path.join(HERE, "_gemm_ref.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", SRC]
    tmp = LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
