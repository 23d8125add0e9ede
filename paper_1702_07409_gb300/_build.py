"""Native build of the package's shared libraries, in-tree.

``libfsgen.so`` (seeded input generator, plain C) is built with gcc;
``libfounsure_gpu.so`` (the C-ABI library and its sm_103a kernels) with nvcc,
one translation unit per process so the compile runs in parallel. Outputs sit
next to their sources and are rebuilt when a source or header is newer.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
GEN_DIR = os.path.join(PKG, "gen")
CSRC = os.path.join(PKG, "csrc")
GEN_LIB = os.path.join(GEN_DIR, "libfsgen.so")
GPU_LIB = os.path.join(CSRC, "libfounsure_gpu.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def _newer(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)


def build_gen(force: bool = False) -> str:
    src = os.path.join(GEN_DIR, "gen.c")
    hdr = os.path.join(INCLUDE, "fs_gen.h")
    if force or _newer(GEN_LIB, [src, hdr]):
        tmp = GEN_LIB + ".tmp%d" % os.getpid()
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-I", INCLUDE, src, "-o", tmp, "-lm"])
        os.replace(tmp, GEN_LIB)
    return GEN_LIB


def _cu_sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def nvcc_path() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def build_gpu(force: bool = False, verbose_ptxas: bool = False) -> str:
    srcs = _cu_sources()
    deps = srcs + _headers()
    if not force and not _newer(GPU_LIB, deps):
        return GPU_LIB
    nvcc = nvcc_path()
    objdir = os.path.join(CSRC, "_build")
    os.makedirs(objdir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def comp(src: str) -> str:
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        _run([nvcc, *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj])
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(comp, srcs))
    tmp = GPU_LIB + ".tmp%d" % os.getpid()
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, GPU_LIB)
    return GPU_LIB


def build_all(force: bool = False) -> None:
    build_gen(force)
    build_gpu(force)
