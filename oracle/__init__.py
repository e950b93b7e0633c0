"""CPU oracle for second-eye synthesis: numpy front end over ``yoro_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
does not import, link or call anything here, and nothing here imports the product.

Each function mirrors one step of the method (Algorithm 1 closed form, Algorithm 2
nearest-wins write, the gather, disocclusion edges, Algorithm 3 with Eq. 6); see
the C source for the definitions and the paper passages they follow.  The submodule
``oracle.unet`` defines the learned hole inpainter (numpy, no C).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "yoro_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_MT_LIB_PATH = os.path.join(_HERE, "liboracle_mt.so")
# binary32 semantics: no contraction of a*b+c into an FMA, no fast-math reassociation.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard"]
_lib = None
_mt_lib = None


def _compile(path: str, extra) -> str:
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, *extra, "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (one thread) and the all-core
    build ``oracle/liboracle_mt.so`` (the same source with -fopenmp: independent rows
    split over the host's cores; the CPU baseline's second leg)."""
    if force:
        for p in (_LIB_PATH, _MT_LIB_PATH):
            if os.path.exists(p):
                os.remove(p)
    _compile(_MT_LIB_PATH, ["-fopenmp"])
    return _compile(_LIB_PATH, [])


def _declare(lib):
    P = ctypes.c_void_p
    I, F = ctypes.c_int, ctypes.c_float
    lib.oracle_disparity.argtypes = [I, I, F, F, F, F, P, P, P]
    lib.oracle_disparity.restype = None
    lib.oracle_forward_warp.argtypes = [I, I, P, P, P, P]
    lib.oracle_forward_warp.restype = None
    lib.oracle_resolve.argtypes = [I, I, P, P, P, P]
    lib.oracle_resolve.restype = None
    lib.oracle_hole_edges.argtypes = [I, I, P, P, P]
    lib.oracle_hole_edges.restype = None
    lib.oracle_fill.argtypes = [I, I, P, P, P, P, P, P]
    lib.oracle_fill.restype = None
    lib.oracle_synthesize.argtypes = [I, I, F, F, F, F, F, F, F, P, P, P, P]
    lib.oracle_synthesize.restype = I
    lib.oracle_fill_ex.argtypes = [I, I, P, P, P, P, P, I, I, P]
    lib.oracle_fill_ex.restype = None
    lib.oracle_synthesize_ex.argtypes = [I, I, F, F, F, F, F, F, F, P, P, I, I, P, P]
    lib.oracle_synthesize_ex.restype = I
    lib.oracle_synthesize_imb.argtypes = [I, I, F, F, F, F, P, P, I, I, I, I, P, P]
    lib.oracle_synthesize_imb.restype = I
    lib.oracle_synthesize_pose.argtypes = [I, I, F, F, F, F, P, P, F, F, P, P, I, I, P, P]
    lib.oracle_synthesize_pose.restype = I
    lib.oracle_threads.argtypes = []
    lib.oracle_threads.restype = I
    return lib


def _load():
    global _lib
    if _lib is None:
        # YORO_ORACLE_LIB names a separately built copy (used by the mutation test).
        _lib = _declare(ctypes.CDLL(os.environ.get("YORO_ORACLE_LIB") or build()))
    return _lib


def _load_mt():
    global _mt_lib
    if _mt_lib is None:
        build()
        _mt_lib = _declare(ctypes.CDLL(_MT_LIB_PATH))
    return _mt_lib


def threads(all_cores: bool = False) -> int:
    """Threads of the one-thread build (1) or of the all-core build."""
    return int((_load_mt() if all_cores else _load()).oracle_threads())


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def disparity(depth, fx, ipd, near, far):
    """Algorithm 1 closed form: (xt int32[H,W] with -1 = off frame, zc float32[H,W])."""
    depth = _c(depth, np.float32)
    h, w = depth.shape
    xt = np.empty((h, w), np.int32)
    zc = np.empty((h, w), np.float32)
    _load().oracle_disparity(w, h, fx, ipd, near, far, depth.ctypes.data, xt.ctypes.data, zc.ctypes.data)
    return xt, zc


def forward_warp(xt, zc):
    """Algorithm 2 nearest-wins write: (src int32[H,W] with -1 = hole, zt float32[H,W])."""
    xt = _c(xt, np.int32)
    zc = _c(zc, np.float32)
    h, w = xt.shape
    src = np.empty((h, w), np.int32)
    zt = np.empty((h, w), np.float32)
    _load().oracle_forward_warp(w, h, xt.ctypes.data, zc.ctypes.data, src.ctypes.data, zt.ctypes.data)
    return src, zt


def resolve(color, src):
    """Gather: (warped uint8[H,W,4] with holes zeroed, mask uint8[H,W] with 1 = hole)."""
    color = _c(color, np.uint8)
    src = _c(src, np.int32)
    h, w = src.shape
    warped = np.empty((h, w, 4), np.uint8)
    mask = np.empty((h, w), np.uint8)
    _load().oracle_resolve(w, h, color.ctypes.data, src.ctypes.data, warped.ctypes.data, mask.ctypes.data)
    return warped, mask


def hole_edges(src):
    """Nearest reached column left (L, -1 if none) and right (R, W if none) of each hole."""
    src = _c(src, np.int32)
    h, w = src.shape
    L = np.empty((h, w), np.int32)
    R = np.empty((h, w), np.int32)
    _load().oracle_hole_edges(w, h, src.ctypes.data, L.ctypes.data, R.ctypes.data)
    return L, R


def fill(src, zt, L, R, warped, kernel_rows=3, nearest_first=False):
    """Algorithm 3 + Eq. 6 over every hole pixel: the final uint8[H,W,4] image.  kernel_rows
    is the kernel height h (odd); nearest_first visits each row's columns from R up."""
    src = _c(src, np.int32)
    zt = _c(zt, np.float32)
    L = _c(L, np.int32)
    R = _c(R, np.int32)
    warped = _c(warped, np.uint8)
    h, w = src.shape
    out = np.empty((h, w, 4), np.uint8)
    _load().oracle_fill_ex(w, h, src.ctypes.data, zt.ctypes.data, L.ctypes.data, R.ctypes.data,
                           warped.ctypes.data, int(kernel_rows), int(bool(nearest_first)), out.ctypes.data)
    return out


def synthesize(color, depth, fx, fy, cx, cy, ipd, near, far, kernel_rows=3, nearest_first=False,
               all_cores=False):
    """Left eye (color uint8[H,W,4], depth float32[H,W]) -> right eye (color, hole mask).
    all_cores runs the all-core build (same arithmetic, rows split over threads)."""
    color = _c(color, np.uint8)
    depth = _c(depth, np.float32)
    h, w = depth.shape
    if color.shape != (h, w, 4):
        raise ValueError("color must be uint8[H,W,4] matching depth")
    out = np.empty((h, w, 4), np.uint8)
    mask = np.empty((h, w), np.uint8)
    lib = _load_mt() if all_cores else _load()
    rc = lib.oracle_synthesize_ex(w, h, fx, fy, cx, cy, ipd, near, far, color.ctypes.data,
                                      depth.ctypes.data, int(kernel_rows), int(bool(nearest_first)),
                                      out.ctypes.data, mask.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_synthesize failed ({rc})")
    return out, mask


def synthesize_imb(color, depth, fx, ipd, near, far, div, interp, kernel_rows=3, nearest_first=False):
    """The path with the row-downsampled intermediate buffer of strategies (c) and (d):
    a reprojection at 1/div of the row resolution (div in 1, 2, 4, 8, 16) and, with
    interp, the shift interpolated between cells and the color sampled linearly."""
    color = _c(color, np.uint8)
    depth = _c(depth, np.float32)
    h, w = depth.shape
    if color.shape != (h, w, 4):
        raise ValueError("color must be uint8[H,W,4] matching depth")
    out = np.empty((h, w, 4), np.uint8)
    mask = np.empty((h, w), np.uint8)
    rc = _load().oracle_synthesize_imb(w, h, fx, ipd, near, far, color.ctypes.data, depth.ctypes.data, int(div),
                                       int(bool(interp)), int(kernel_rows), int(bool(nearest_first)),
                                       out.ctypes.data, mask.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_synthesize_imb failed ({rc})")
    return out, mask


def synthesize_pose(color, depth, fx, fy, cx, cy, rot, c, near, far, kernel_rows=3, nearest_first=False):
    """The path with a general second-eye pose (Eq. 5 with a general M): rotation rot
    (3x3, p' = rot (p - c)) and position c (3) of the second eye in left-eye camera
    coordinates; pixels may leave their row."""
    color = _c(color, np.uint8)
    depth = _c(depth, np.float32)
    rot = _c(rot, np.float32).reshape(9)
    c = _c(c, np.float32).reshape(3)
    h, w = depth.shape
    if color.shape != (h, w, 4):
        raise ValueError("color must be uint8[H,W,4] matching depth")
    out = np.empty((h, w, 4), np.uint8)
    mask = np.empty((h, w), np.uint8)
    rc = _load().oracle_synthesize_pose(w, h, fx, fy, cx, cy, rot.ctypes.data, c.ctypes.data, near, far,
                                        color.ctypes.data, depth.ctypes.data, int(kernel_rows),
                                        int(bool(nearest_first)), out.ctypes.data, mask.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_synthesize_pose failed ({rc})")
    return out, mask


def synthesize_steps(color, depth, fx, ipd, near, far):
    """The path step by step, returning every intermediate (for tests)."""
    xt, zc = disparity(depth, fx, ipd, near, far)
    src, zt = forward_warp(xt, zc)
    warped, mask = resolve(color, src)
    L, R = hole_edges(src)
    out = fill(src, zt, L, R, warped)
    return dict(xt=xt, zc=zc, src=src, zt=zt, warped=warped, mask=mask, L=L, R=R, out=out)
