"""Builds the CUDA extension libqedm2.so in-tree for sm_103a with nvcc.

Two steps: the DAG builder's code generator (csrc/qed_codegen.cpp, compiled
with g++ against csrc/dag.cpp) writes the straight-line specialised forward
kernels into _build/qed_spec_gen.cu; nvcc then compiles every source and that
file (one object each, in parallel, under _build/) and links one shared
library.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqedm2.so")
GEN = os.path.join(BUILD, "qed_spec_gen.cu")
SOURCES = ["dag.cpp", "qed_api.cpp", "qed_fwd.cu", "qed_rw.cu", "abc_kernel.cu", "qed_tape.cu", "qed_adj.cu",
           "qed_batch.cu", "qed_noalloc.cu", "qed_gen.cu", "qed_peak.cu", "qed_fix.cu", "qed_radj.cu"]
HEADERS = ["dag.hpp", "qed_types.h", "qed_device.cuh", "qed_team.cuh", "qed_eval.cuh", "qed_plan.hpp", "qed_batch.cuh",
           "qed_spec.cuh", "qed_adjoint.cuh"]
GENERATOR = ["qed_codegen.cpp", "dag.cpp", "dag.hpp", "qed_types.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _mtime(p: str) -> float:
    return os.path.getmtime(p) if os.path.exists(p) else -1.0


def _headers_mtime() -> float:
    return max(_mtime(os.path.join(CSRC, h)) for h in HEADERS + ["../../include/qed.h"])


def generate() -> str:
    """Compiles and runs the code generator; returns the generated source."""
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "qed_codegen")
    if _mtime(exe) < max(_mtime(os.path.join(CSRC, f)) for f in GENERATOR):
        cxx = os.environ.get("CXX", "g++")
        subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(CSRC, "qed_codegen.cpp"),
                               os.path.join(CSRC, "dag.cpp"), "-o", exe + ".tmp"])
        os.replace(exe + ".tmp", exe)
    subprocess.check_call([exe, GEN])   # rewrites GEN only when its text changes
    return GEN


def _objects(sources, verbose):
    nvcc = os.environ.get("NVCC", "nvcc")
    hdr = _headers_mtime()
    jobs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if _mtime(obj) < max(_mtime(src), hdr):
            cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj + ".tmp"]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((cmd, obj))
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        for (cmd, obj), fut in zip(jobs, [ex.submit(subprocess.check_call, c) for c, _ in jobs]):
            fut.result()
            os.replace(obj + ".tmp", obj)
    return [os.path.join(BUILD, os.path.basename(s) + ".o") for s in sources]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    gen = generate()
    sources = [os.path.join(CSRC, f) for f in SOURCES] + [gen]
    if force:
        for s in sources:
            o = os.path.join(BUILD, os.path.basename(s) + ".o")
            if os.path.exists(o):
                os.remove(o)
    objs = _objects(sources, verbose)
    if force or _mtime(LIB) < max(_mtime(o) for o in objs):
        nvcc = os.environ.get("NVCC", "nvcc")
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call([nvcc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


def _stale() -> bool:
    """True when build() would recompile or relink (without running it)."""
    gen_inputs = max(_mtime(os.path.join(CSRC, f)) for f in GENERATOR)
    srcs = [os.path.join(CSRC, f) for f in SOURCES]
    newest = max([_headers_mtime(), gen_inputs] + [_mtime(s) for s in srcs])
    return _mtime(LIB) < newest


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
