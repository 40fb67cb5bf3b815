"""TEST INFRASTRUCTURE ONLY: compiles the oracle's C bilateral filter with the host gcc.

``build()`` writes ``oracle/_build/liboracle_blf.so``.  Plain ``-O2`` (no fast-math) keeps
libm's FP64 ``exp`` and IEEE evaluation order; OpenMP spreads rows over the host cores.  The
flags carry nothing machine-specific, so the same command builds on x86-64 and on AArch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "blf_ref.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_blf.so")


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
