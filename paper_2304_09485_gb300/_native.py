"""Build and load libhgks.so (in-tree, sm_103a).

The library is compiled from csrc/ with nvcc for sm_103a only; translation
units are compiled in parallel and linked into _build/libhgks.so. Loading
fails loudly when the library is missing or cannot be opened: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhgks.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["residual.cu", "implicit.cu", "batch.cu", "batch_capi.cu", "server.cu", "capi.cu", "noalloc.cu", "peak.cu", "mesh_setup.cpp"]
HEADERS = ["hgks_internal.h", "givens.cuh", "offdiag.cuh", "batch_impl.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in ("nvcc", "/usr/local/cuda/bin/nvcc"):
        try:
            subprocess.run([c, "--version"], capture_output=True, check=True)
            return c
        except (OSError, subprocess.CalledProcessError):
            pass
    raise RuntimeError("nvcc not found: libhgks cannot be built")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "hgks.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile libhgks.so for sm_103a (nvcc, -O3, -lineinfo)."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-I", INCLUDE, "-Xcompiler", "-fPIC"]
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + ARCH + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "c++"] + common + ["-Xcompiler", "-ffp-contract=off,-pthread", "-c",
                                                  os.path.join(CSRC, src), "-o", obj]
        elif ptxas_info:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-Xcompiler", "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


_lib = None


def load() -> ctypes.CDLL:
    """Open libhgks.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = build()
        _lib = ctypes.CDLL(path)
    return _lib
