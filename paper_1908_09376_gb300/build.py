"""Builds the in-tree shared library libmidbf.so (host C++ + CUDA for sm_103a).

Run as ``python paper_1908_09376_gb300/build.py`` (a plain script: importing the
package would load the library it builds) or through ``__graft_entry__.build()``.
Host sources compile with g++, CUDA sources with nvcc
(-gencode arch=compute_103a,code=sm_103a), in parallel; nvcc links the
result against the CUDA runtime.  Objects go to ``_build/`` next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmidbf.so")

HOST = ["capi.cpp", "phase.cpp", "plan.cpp", "qr.cpp", "build.cpp", "recover.cpp"]
CUDA = ["device.cu", "launch_rc.cu", "launch_s.cu", "launch_tc.cu", "batched.cu", "build_gpu.cu", "recover_gpu.cu",
        "measure.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "midbf.h"))
    jobs, objs = [], []
    for f in HOST:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            jobs.append(["g++", "-std=c++17", "-O3", "-fPIC", "-pthread", "-fcx-limited-range",
                         "-Wall", "-Wno-unused-function", "-c", src, "-o", obj])
    for f in CUDA:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-pthread",
                   "-c", src, "-o", obj]
            if ptxas_verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(_run, jobs):
            if verbose and out.strip():
                print(out)
    if jobs or not os.path.exists(LIB):
        _run([nvcc, "-shared", *ARCH, "-o", LIB, *objs, "-lpthread"])
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_verbose="-v" in sys.argv))
