"""Builds librr.so in-tree for sm_103a (nvcc, no cmake).

Every translation unit under csrc/ is compiled in parallel into _build/ and
linked, with the static CUDA runtime, into paper_2506_11273_gb300/librr.so,
and once more with RR_CHECKED (every kernel index checked against its buffer)
into _build_checked/ and librr_checked.so.
A unit is rebuilt when it or any header under csrc/ or include/ is newer
than its object file.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB = os.path.join(PKG, "librr.so")
LIB_CHECKED = os.path.join(PKG, "librr_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr", "-I", INCLUDE]
CXX_FLAGS = ["-O3", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librr")


def _cuda_include() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(_nvcc()))), "include")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(src: str, obj: str, newest_header: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or newest_header > t


def _build_one(build_dir: str, lib: str, defines, verbose: bool, ptxas_info: bool, force: bool):
    """Compiles every unit into build_dir and returns (lib, link command or None,
    running compiler processes)."""
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    newest = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    procs = []
    objs = []
    for src in sources:
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        if not force and not _stale(src, obj, newest):
            continue
        if src.endswith(".cu"):
            cmd = [nvcc] + ARCH + NVCC_FLAGS + defines + (["-Xptxas", "-v"] if ptxas_info else []) + \
                ["-c", src, "-o", obj]
        else:
            cmd = ["g++"] + CXX_FLAGS + defines + ["-I", _cuda_include(), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    link = None
    if procs or not os.path.exists(lib):
        tmp = lib + ".%d.tmp" % os.getpid()
        link = ([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"], tmp)
    return link, procs


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False) -> str:
    """Builds librr.so and its bounds-checked twin librr_checked.so (every
    kernel index checked against its buffer, RR_CHECKED); the units of both
    compile in parallel."""
    jobs = [(LIB, _build_one(BUILD, LIB, [], verbose, ptxas_info, force)),
            (LIB_CHECKED, _build_one(BUILD_CHECKED, LIB_CHECKED, ["-DRR_CHECKED"], verbose, False, force))]
    failed = []
    for _, (_, procs) in jobs:
        for src, p in procs:
            out, _ = p.communicate()
            text = out.decode(errors="replace")
            if p.returncode != 0:
                failed.append((src, text))
            elif verbose or ptxas_info:
                sys.stderr.write(text)
    if failed:
        msg = "\n".join("%s:\n%s" % (s, t) for s, t in failed)
        raise RuntimeError("librr build failed\n" + msg)
    for lib, (link, _) in jobs:
        if link is None:
            continue
        cmd, tmp = link
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv, force="-f" in sys.argv)
    print(LIB)
