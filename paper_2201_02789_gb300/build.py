"""Builds the CUDA library ``_build/libnestpar.so`` for sm_103a.

Each translation unit under ``csrc/`` is compiled with relocatable device code
(device-side launches need it) in parallel, then linked with the device
runtime (``cudadevrt``) into one shared library. No cmake.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libnestpar.so")
SOURCES = ["np_capi.cu", "np_engine.cu", "np_batch.cu", "np_server.cu", "np_bfs.cu", "np_sssp.cu", "np_bezier.cu",
           "np_tc.cu", "np_sssp64.cu", "np_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-rdc=true", "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnestpar")
    return path


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h", ".map"))]
    files.append(os.path.join(INCLUDE, "nestpar.h"))
    return files


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, defines: tuple[str, ...] = (), out_dir: str | None = None) -> str:
    """Compile and link if any source changed; returns the library path.

    ``defines`` (``NAME=VALUE`` strings) and ``out_dir`` build a variant of the
    library elsewhere, for tuning experiments; the default build uses neither."""
    bdir = out_dir or BUILD
    lib = os.path.join(bdir, "libnestpar.so")
    if out_dir is None and not force and not stale():
        return LIB
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    dflags = ["-D" + d for d in defines]

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *CFLAGS, *dflags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    # export the C ABI only: the statically linked CUDA runtime stays private, so
    # it can never be interposed by another runtime loaded in the same process
    cmd = [cc, *ARCH, "-shared", "-rdc=true", "-Xcompiler", "-fPIC",
           "-Xlinker", "--version-script=" + os.path.join(CSRC, "exports.map"),
           "-o", tmp, *objs, "-lcudadevrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))


GEN_SRC = os.path.join(PKG, "gen_native.c")
GEN_LIB = os.path.join(BUILD, "libnpgen.so")


def build_gen(force: bool = False) -> str:
    """Compile the C twin of the input generator (gen_native.c) with gcc."""
    if not force and os.path.exists(GEN_LIB) and os.path.getmtime(GEN_LIB) >= os.path.getmtime(GEN_SRC):
        return GEN_LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = GEN_LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", GEN_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed on gen_native.c:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, GEN_LIB)
    return GEN_LIB
