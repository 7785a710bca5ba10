"""Build the sm_103a shared library libmm.so in-tree (paper_1005_5198_gb300/_build).

nvcc compiles the CUDA translation unit for sm_103a only, g++ the host runtime
(plain IEEE arithmetic: no FMA contraction, so the seeded lens fields match
other implementations bit for bit); the units compile in parallel and link
into one shared library with the CUDA runtime linked statically.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmm.so")
ALU_RATES = os.path.join(BUILD, "alu_rates")     # pipe-throughput probe, built only on request (build_alu_rates)
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["mm_fp64.cu", "mm_fp32_c1r8.cu", "mm_fp32_c2r4.cu", "mm_fp32_c2r8.cu", "mm_fp32_c2r4w.cu", "mm_fp32_random.cu",
              "mm_noalloc.cu", "mm_stats.cu", "mm_extended.cu", "mm_far.cu", "mm_tree.cu"]
CPP_SOURCES = ["mm_host.cpp", "mm_serve.cpp"]
HEADERS = ["mm_internal.h", "mm_ctx.h", "mm_device.cuh", "mm_fp32.cuh", "mm_far.h"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "mm.h"))
    files.append(os.path.abspath(__file__))
    return files


# Checked build (-DMM_CHECKS): every guarded device access tests its index and a
# failure comes back as MM_EDEVICE instead of a fault; for debugging, not timing.
CHECKED_BUILD = os.path.join(BUILD, "checked")
CHECKED_LIB = os.path.join(CHECKED_BUILD, "libmm.so")


def up_to_date(checked: bool = False) -> bool:
    outs = [CHECKED_LIB] if checked else [LIB]
    if not all(os.path.exists(o) for o in outs):
        return False
    t = min(os.path.getmtime(o) for o in outs)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib_path = CHECKED_LIB if checked else LIB
    if not force and up_to_date(checked):
        return lib_path
    out_dir = CHECKED_BUILD if checked else BUILD
    os.makedirs(out_dir, exist_ok=True)
    defs = ["-DMM_CHECKS"] if checked else []
    jobs, objs = [], []
    for f in CU_SOURCES:
        o = os.path.join(out_dir, f + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v", *defs,
               "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append((f, cmd))
        objs.append(o)
    for f in CPP_SOURCES:
        o = os.path.join(out_dir, f + ".o")
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall", "-Wextra", *defs,
               "-I", os.path.join(CUDA_HOME, "include"), "-I", os.path.join(ROOT, "include"),
               "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append((f, cmd))
        objs.append(o)
    procs = [(f, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)) for f, c in jobs]
    logs = []
    for f, p in procs:
        out, _ = p.communicate()
        logs.append((f, out))
        if p.returncode != 0:
            raise RuntimeError(f"compiling {f} failed:\n{out}")
    tmp = lib_path + f".{os.getpid()}.tmp"
    link = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking libmm.so failed:\n{r.stdout}")
    os.replace(tmp, lib_path)
    with open(os.path.join(out_dir, "ptxas.log"), "w") as fh:
        for f, out in logs:
            fh.write(f"== {f}\n{out}\n")
    if verbose:
        for f, out in logs:
            sys.stdout.write(f"== {f}\n{out}\n")
    return lib_path


def build_alu_rates() -> str:
    """Compile the arithmetic-pipe probe (alu_rates.cu: FFMA, FFMA2, MUFU and DFMA rates per SM per
    clock, and the shooting kernel's instruction mix) as a standalone program. It measures the
    roofline's denominators and is not part of libmm.so."""
    src = os.path.join(CSRC, "alu_rates.cu")
    os.makedirs(BUILD, exist_ok=True)
    if os.path.exists(ALU_RATES) and os.path.getmtime(ALU_RATES) >= os.path.getmtime(src):
        return ALU_RATES
    tmp = ALU_RATES + f".{os.getpid()}.tmp"
    subprocess.run([NVCC, *ARCH, "-O3", "-std=c++17", src, "-o", tmp], check=True)
    os.replace(tmp, ALU_RATES)
    return ALU_RATES


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
