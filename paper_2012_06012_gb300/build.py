"""Builds libmgt.so (the C-ABI library with the sm_103a kernels) in-tree.

Each .cu translation unit is compiled by nvcc in parallel, then linked into
``paper_2012_06012_gb300/libmgt.so``.  No cmake; only nvcc and the host
compiler.  Re-running is cheap: units whose object is newer than every
source and header are skipped.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
DEBUG = os.environ.get("MGT_DEBUG") == "1"
BUILD = os.path.join(HERE, "_build_debug" if DEBUG else "_build")
LIB = os.path.join(HERE, "libmgt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(debug: bool) -> list[str]:
    f = ARCH + ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                f"-I{os.path.join(ROOT, 'include')}", "--expt-relaxed-constexpr"]
    if debug:
        f += ["-DMGT_DEBUG=1"]
    return f


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + [
        os.path.join(ROOT, "include", "mgt.h"), __file__]
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def build(force: bool = False, verbose: bool = False, debug: bool = DEBUG,
          ptxas_info: bool = False) -> str:
    """debug=True (or MGT_DEBUG=1) compiles the bounds-checked variant of the
    kernels into a separate object folder; the library path is the same."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    dep = _deps_mtime()
    jobs = []
    objs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        if (force or ptxas_info or not os.path.exists(obj)
                or os.path.getmtime(obj) < max(dep, os.path.getmtime(src))):
            cmd = [nvcc] + _flags(debug) + ["-c", src, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [nvcc, "-x", "cu"] + cmd[1:]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or ptxas_info or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3] if not ptxas_info else cmd}")
    if jobs or force or not os.path.exists(LIB) or debug != _lib_is_debug():
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "shared", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link of libmgt.so failed")
        os.replace(tmp, LIB)
        with open(LIB + ".flavor", "w") as f:
            f.write("debug" if debug else "release")
    return LIB


def _lib_is_debug() -> bool:
    try:
        with open(LIB + ".flavor") as f:
            return f.read().strip() == "debug"
    except OSError:
        return False


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
