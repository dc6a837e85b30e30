"""Build the CUDA library libqbx_gb300.so in-tree (paper_1207_4461_gb300/_build/).

nvcc compiles each translation unit for sm_103a in parallel, then links one
shared library with the C ABI of include/qbx.h.  No cmake, no torch extension
machinery: the library has no torch types in its interface.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libqbx_gb300.so")
SOURCES = ["qbx_apply_real.cu", "qbx_apply_cplx.cu", "qbx_apply_local.cu", "qbx_far.cu", "qbx_misc.cu", "qbx_capi.cu", "qbx_batch.cu",
           "qbx_adjoint.cu", "qbx_gmres.cu", "qbx_shape.cu", "qbx_assemble.cu",
           "qbx_static.cu", "qbx_grad_d.cu", "qbx_hk_table.cu", "qbx_zgemm.cu"]
HEADERS = ["qbx_device.cuh", "qbx_internal.h", "special_tables.h", "qbx_apply_impl.cuh",
           "qbx_group_impl.cuh", "qbx_adjoint_impl.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose_ptx: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]
    if verbose_ptx:
        f += ["-Xptxas", "-v"]
    return f


def _stale(lib: str, deps) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptx: bool = False, quiet: bool = True) -> str:
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [
        os.path.join(HERE, "..", "include", "qbx.h"), os.path.abspath(__file__)]
    if not force and not _stale(LIB, deps):
        return LIB
    nv = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nv] + _flags(verbose_ptx) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose_ptx or not quiet:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nv] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptx="-v" in sys.argv, quiet=False))
