"""Build of the CUDA library ``libyoro.so`` (sm_103a) and the host-side C pieces.

Each ``.cu`` translation unit is compiled by nvcc in parallel, then linked into a
shared library in ``paper_2506_15183_gb300/_lib/``; object files go to ``_build/``.
Flags: ``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3 -fmad=false`` (no
contraction of separate multiplies and adds into FMAs; the kernels also spell
every float operation with round-to-nearest intrinsics), no fast-math, so
denormals are kept and division is IEEE.

``build_cuda(debug=True)`` builds the debug-bounds variant ``libyoro_debug.so`` from
the same sources with ``-DYORO_DEBUG_BOUNDS`` (objects in ``_build/debug/``): every
computed shared- or global-memory index is range-checked, a failing access is skipped
and recorded in a device status word that ``yoro_stream_status`` reports.  It is built
on demand only, never by ``build_all``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libyoro.so")
DEBUG_LIB = os.path.join(LIBDIR, "libyoro_debug.so")
SOURCES = ["api.cu", "fused.cu", "unfused.cu", "noalloc.cu", "server.cu", "imbuffer.cu", "pose.cu", "unet.cu", "unet_train.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
              "-Xptxas", "-v", f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libyoro.so")


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files.append(__file__)
    return max(os.path.getmtime(f) for f in files if os.path.isfile(f))


def _compile(src: str, debug: bool = False) -> tuple[str, str]:
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
    extra = ["-DYORO_DEBUG_BOUNDS"] if debug else []
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build_cuda(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libyoro.so (or, with debug, libyoro_debug.so) if any source is
    newer than it; returns its path."""
    lib = DEBUG_LIB if debug else LIB
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _inputs_mtime():
        return lib
    os.makedirs(bdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda src: _compile(src, debug), SOURCES))
    log = "\n".join(err for _, err in results)
    with open(os.path.join(bdir, "ptxas.log"), "w") as fh:
        fh.write(log)
    if verbose:
        print(log)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> None:
    """The CUDA library and the scene generator (host C)."""
    from .scene import build as build_scene

    build_scene(force=force)
    build_cuda(force=force, verbose=verbose)


if __name__ == "__main__":
    build_all(force=True, verbose=True)
