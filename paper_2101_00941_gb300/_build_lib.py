"""Build of libdd.so: nvcc for sm_103a, one object per translation unit, compiled in parallel."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD, "libdd.so")
SOURCES = ("dd_api.cu", "dd_kernels.cu", "dd_dedisp.cu", "dd_static.cu", "dd_serve.cu", "dd_batch.cu",
           "dd_peaks.cu", "dd_group.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code without floating-point contraction: FP64 host arithmetic (candidate DMs) rounds once
# per operation on x86 and Arm alike
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-ffp-contract=off",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu into _build/libdd.so (skipped when up to date)."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, "dd_internal.h"), os.path.join(ROOT, "include", "dd.h"),
                   os.path.join(CSRC, "dd_dedisp.cuh")]
    deps = [d for d in deps if os.path.exists(d)]
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return LIB_PATH
    nvcc = _nvcc()
    objs, procs = [], []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + f".{os.getpid()}.o")
        objs.append(o)
        cmd = [nvcc, *ARCH, *FLAGS, "-c", s, "-o", o]
        if verbose:
            cmd.append("-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            errs.append(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        if pr.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    if verbose and errs:
        print("\n".join(errs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                           "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-Xlinker", "-z,defs"])
    os.replace(tmp, LIB_PATH)
    for o in objs:
        os.remove(o)
    return LIB_PATH
