"""Builds libqaoa.so in-tree for sm_103a.

Host C++ translation units are compiled with g++, CUDA ones with nvcc
(``-gencode arch=compute_103a,code=sm_103a -lineinfo``), all in parallel,
then linked with nvcc into ``paper_2101_10296_gb300/libqaoa.so`` (CUDA
runtime linked statically, so the library has no dependency beyond the
driver).  Objects go to ``paper_2101_10296_gb300/_build/``.

Run ``python -m paper_2101_10296_gb300.build`` (or call :func:`build`).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqaoa.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SRC = ["graph.cpp", "orbits.cpp", "plan.cpp", "cone_classes.cpp", "block_orbits.cpp"]
CUDA_SRC = ["kernels.cu", "kernels_grad.cu", "kernels_grad5.cu", "big.cu", "big_split.cu", "capi.cu", "noalloc.cu", "p1_kernel.cu"]
HEADERS = ["host.hpp", "device.cuh", "big.cuh", "big_common.cuh", "devplan.cuh", "cone_kernel.cuh", "dev_math.cuh",
           "kernels_grad_impl.cuh", "reg_common.cuh"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _commands(verbose_ptxas=False):
    nvcc = _nvcc()
    cmds = []
    for src in HOST_SRC:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmds.append((obj, ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function",
                           "-I", ROOT, "-c", os.path.join(CSRC, src), "-o", obj]))
    for src in CUDA_SRC:
        obj = os.path.join(OUT_DIR, src + ".o")
        flags = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
                 "-Xcompiler", "-fPIC", "-I", ROOT, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose_ptxas:
            flags.insert(1, "-Xptxas=-v")
        cmds.append((obj, flags))
    return cmds


def _stale(obj, src_paths):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in src_paths)


def build(force=False, verbose_ptxas=False, quiet=True):
    """Compile every translation unit (in parallel) and link libqaoa.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "qaoa.h")]
    procs = []
    objs = []
    for obj, cmd in _commands(verbose_ptxas):
        src = cmd[cmd.index("-c") + 1]
        objs.append(obj)
        if force or verbose_ptxas or _stale(obj, [src] + deps):
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, pr in procs:
        out, _ = pr.communicate()
        text = out.decode(errors="replace")
        if pr.returncode != 0:
            failed.append((cmd, text))
        elif text.strip() and not quiet:
            sys.stderr.write(text)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("libqaoa build failed:\n" + msg)
    if force or procs or not os.path.exists(LIB) or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("libqaoa link failed:\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False)
    print(LIB)
