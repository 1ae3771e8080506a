"""Compile the CPU oracle (plain C, FP64, OpenMP) into oracle/liboracle.so and
the CPU segment-tree baseline into oracle/libsegtree.so.

Test infrastructure: both are built here so that the checker and the CPU
baseline exist on any machine with gcc; building them is not using them.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "egm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
SEG_SRC = os.path.join(HERE, "segtree.c")
SEG_LIB = os.path.join(HERE, "libsegtree.so")

# -ffp-contract=off: every expression is rounded as written (no fused multiply-add).
CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared", "-Wall", "-Wextra"]
# the baseline is timed: optimised, but with the same rounding rules
SEG_CFLAGS = ["-O3", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
              "-fPIC", "-shared", "-Wall", "-Wextra"]


def _compile(src, lib, flags, force):
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *flags, src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    _compile(SEG_SRC, SEG_LIB, SEG_CFLAGS, force)
    return _compile(SRC, LIB, CFLAGS, force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
