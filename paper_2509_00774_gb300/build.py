"""Build the CUDA library libnfmimo.so in-tree for sm_103a with nvcc.

The translation units compile in parallel; the result is
paper_2509_00774_gb300/libnfmimo.so (git-ignored).  Only the CUDA runtime is
linked (statically), so the library needs no PyTorch.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnfmimo.so")
SOURCES = ["nfm_api.cu", "op_forward.cu", "op_adjoint.cu", "op_adjoint_tc.cu", "op_misc.cu", "op_prox.cu", "op_general.cu",
           "op_cheb.cu", "op_cheb_tc.cu", "op_cheb_tc_fwd.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# per-file extra flags: the expansion kernels handle no subnormal values (distances, unit phasors,
# Chebyshev values in [-1, 1]); flushing them lets rsqrt / reciprocal skip their subnormal paths
FILE_FLAGS = {"op_cheb.cu": ["-ftz=true"], "op_cheb_tc.cu": ["-ftz=true"], "op_cheb_tc_fwd.cu": ["-ftz=true"]}
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "nfmimo.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


LIB_CHECK = os.path.join(HERE, "libnfmimo_check.so")


def build(force: bool = False, verbose: bool = False, extra_flags=None, check: bool = False) -> str:
    """Build libnfmimo.so, or with check=True the bounds-checked libnfmimo_check.so (-DNFM_BOUNDS_CHECK:
    checked kernel indices raise a device flag instead of leaving their buffer)."""
    lib, bdir = (LIB_CHECK, BUILD + "_check") if check else (LIB, BUILD)
    if not force and os.path.exists(lib) and all(os.path.getmtime(f) <= os.path.getmtime(lib) for f in _deps()):
        return lib
    os.makedirs(bdir, exist_ok=True)
    flags = NVCC_FLAGS + list(extra_flags or []) + (["-DNFM_BOUNDS_CHECK"] if check else [])

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc()] + ARCH + flags + FILE_FLAGS.get(src, []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
