"""Build the RBE C-ABI shared library (librbe_gb300.so) for sm_103a with nvcc.

Each CUDA translation unit compiles in parallel; the objects link into one shared
library next to this file (`_build/`). The build is in-tree and needs no cmake.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librbe_gb300.so")
SOURCES = ["rbe_api.cu", "k_sample.cu", "k_bin.cu", "k_kspace.cu", "k_pair.cu", "k_rbl.cu",
           "k_integrate.cu", "rbe_noalloc.cu", "k_probe.cu", "k_list.cu", "k_cpair.cu",
           "k_coul.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit multiply-add contraction; the kernels write every fused
# multiply-add out (fmaf / fma), so any two compilations of a kernel body (a replica's own
# launch and the batched launch over many replicas) round alike and agree bit for bit.
# Files whose kernels have no batched copy may let the compiler contract: k_pair.cu (the
# per-particle pair kernel, one launch per replica; its FP64 instance, the FP64 form's pair
# pass, runs 6% faster so). The cutoff decisions there are written with explicit roundings.
CONTRACT = {"k_pair.cu"}
NVCC_FLAGS = ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdrs + [os.path.join(INCLUDE, "rbe.h"), os.path.abspath(__file__)]


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile every translation unit and link the shared library; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    dep_time = max(os.path.getmtime(p) for p in _deps() + srcs)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= dep_time:
        return LIB
    cc = nvcc()
    extra = list(extra or [])
    procs = []
    objs = []
    for src in srcs:
        obj = os.path.join(OUT_DIR, os.path.basename(src).replace(".cu", ".o"))
        objs.append(obj)
        flags = list(NVCC_FLAGS)
        if os.path.basename(src) in CONTRACT:
            flags = [f if f != "-fmad=false" else "-fmad=true" for f in flags]
        cmd = [cc, *ARCH, *flags, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or (verbose and out):
            sys.stderr.write(out.decode(errors="replace"))
        if pr.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
