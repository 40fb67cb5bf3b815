"""Build ``libblfls.so`` (the C-ABI library) in-tree with nvcc for sm_103a.

Every translation unit under ``csrc/`` is compiled in parallel into ``_build/obj`` and linked into
``_build/libblfls.so`` (CUDA runtime linked statically).  Objects are rebuilt only when a source
or header is newer.  Runs the same way on an x86-64 host (cross-compiling, no GPU needed) and on
an AArch64 GPU host.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libblfls.so")
# The debug build: device range checks compiled in (-DBLFLS_DEVICE_CHECKS, see csrc/dcheck.cuh),
# in a directory of its own so that it never replaces the release library.
DEBUG_OUT = os.path.join(OUT, "debug")
DEBUG_LIB = os.path.join(DEBUG_OUT, "libblfls.so")
DEBUG_FLAGS = ["-DBLFLS_DEVICE_CHECKS"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers() -> list[str]:
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _compile(src: str, obj: str, extra: list[str]) -> tuple[str, int, str]:
    cmd = [nvcc()] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    return src, p.returncode, p.stdout + p.stderr


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None,
          debug: bool = False) -> str:
    """Compile and link the library (the debug build with `debug`); return its path.  Raises
    RuntimeError on failure."""
    out_dir, lib_path = (DEBUG_OUT, DEBUG_LIB) if debug else (OUT, LIB)
    flags = list(extra or []) + (DEBUG_FLAGS if debug else [])
    os.makedirs(os.path.join(out_dir, "obj"), exist_ok=True)
    newest_hdr = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    jobs = []
    objs = []
    for src in _sources():
        obj = os.path.join(out_dir, "obj", os.path.basename(src) + ".o")
        objs.append(obj)
        stale = (force or extra or not os.path.exists(obj)
                 or os.path.getmtime(obj) < max(os.path.getmtime(src), newest_hdr))
        if stale:
            jobs.append((src, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for src, rc, log in ex.map(lambda j: _compile(j[0], j[1], flags), jobs):
                if verbose or rc != 0:
                    sys.stderr.write(log)
                if rc != 0:
                    raise RuntimeError(f"nvcc failed on {os.path.basename(src)}")
    if jobs or not os.path.exists(lib_path):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            sys.stderr.write(p.stdout + p.stderr)
            raise RuntimeError("link of libblfls.so failed")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="--force" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None,
                debug="--debug" in sys.argv))
