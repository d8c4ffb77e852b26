"""Build libsimplets.so (the C-ABI library of include/simplets.h) in-tree with
nvcc for sm_103a.  Translation units compile in parallel; no cmake."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsimplets.so")
SOURCES = ["phase_df64.cu", "step_df64.cu", "phase_fp64.cu", "step_fp64.cu", "phase_mixed.cu", "step_mixed.cu",
           "sweep_kernels.cu", "persistent.cu", "simplets_host.cu", "alu_probe.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The FP32 and double-float kernels are compiled without multiply-add
# contraction: every FP32 operation is rounded as written (the FMAs they need
# are explicit), so each compiled form of a body -- descriptor read in place
# or staged, per-phase or persistent -- gives the same bits.  The FP64 kernels
# keep it: they are bound by the FP64 pipe, where each fused pair saves an
# instruction, and all their forms stage the descriptor the same way.
EXTRA_FLAGS = {f: ["--fmad=false"] for f in ("phase_mixed.cu", "step_mixed.cu", "phase_df64.cu", "step_df64.cu")}


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsimplets.so")
    return exe


def _flags():
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _newest_input() -> float:
    inc = os.path.join(ROOT, "include")
    paths = ([os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(inc, f) for f in os.listdir(inc)]
             + [os.path.abspath(__file__)])
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [exe, *_flags(), *EXTRA_FLAGS.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    # the shared CUDA runtime: one runtime instance per process, the same one
    # PyTorch uses when both are loaded
    cudart_dir = os.path.join(os.path.dirname(os.path.dirname(exe)), "lib64")
    r = subprocess.run([exe, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", f"-rpath,{cudart_dir}",
                        "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
