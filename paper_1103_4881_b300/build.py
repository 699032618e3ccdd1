"""Build libds.so (the CUDA library) in-tree with nvcc for sm_103a, and
libds_check.so, the same sources with -DDS_CHECK_BOUNDS (the fused kernel
checks its own indices and reports a failure instead of making the access).

Usage: python -m paper_1103_4881_b300.build [--force] [--verbose] [--check]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libds.so")
CHECK_LIB = os.path.join(HERE, "libds_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "ds.h"), os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False, check_bounds: bool = False) -> str:
    """Compile every source under csrc/ into paper_1103_4881_b300/libds.so
    (check_bounds: libds_check.so, with -DDS_CHECK_BOUNDS)."""
    lib = CHECK_LIB if check_bounds else LIB
    if not force and up_to_date(lib):
        return lib
    objdir = os.path.join(HERE, "_build_check" if check_bounds else "_build")
    os.makedirs(objdir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH
    if check_bounds:
        common += ["-DDS_CHECK_BOUNDS"]
    if verbose:
        common += ["-Xptxas", "-v"]
    objs = []
    procs = []
    # an object is rebuilt when it is older than its source or any header
    headers = [p for p in _inputs() if not p.endswith((".cu", ".cpp"))]
    newest_header = max(os.path.getmtime(p) for p in headers)
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header):
            continue
        cmd = [nvcc()] + common + ["-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + text)
        failed |= p.returncode != 0
    if failed:
        raise RuntimeError("nvcc failed building libds")
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, check_bounds="--check" in sys.argv))
