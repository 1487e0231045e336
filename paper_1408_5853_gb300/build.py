"""Build the CUDA library ``_build/libccell.so`` (sm_103a) in-tree with nvcc."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libccell.so")
SOURCES = ["ccell_step.cu", "ccell_step_persist.cu", "ccell_step_mixed.cu",
           "ccell_step_mixed_persist.cu", "ccell_adjoint.cu", "ccell_api.cpp", "ccell_noalloc.cu",
           "ccell_powtab.cpp", "ccell_adi.cu", "ccell_grid.cpp",
           "ccell_fp64_rate.cu", "ccell_step_lines.cu",
           "ccell_step_lines_mixed.cu", "ccell_step_resident.cu",
           "ccell_step_pipe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HEADERS = ["ccell_internal.h", "ccell_host.h", "ccell_device.cuh", "ccell_fp64_task.cuh", "ccell_mixed_task.cuh",
           "ccell_lines.cuh", "ccell_lines_mixed.cuh",
           os.path.join("..", "..", "include", "ccell.h")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libccell")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit for sm_103a and link the shared library."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", os.path.join(HERE, "..", "include")]
    common += os.environ.get("CCELL_NVCC_EXTRA", "").split()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc] + common + (["-Xptxas", "-v"] if verbose else []) + [
            "-x", "cu" if src.endswith(".cu") else "c++", "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        if verbose:
            print(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    res = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
