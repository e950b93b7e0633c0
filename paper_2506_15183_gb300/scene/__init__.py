"""Seeded synthetic scenes ray-cast on the host: the inputs of second-eye synthesis.

This module is input generation only.  It renders an eye of a procedural scene
(spheres and axis-aligned boxes, optional checkered ground plane, Lambert shading)
to RGBA8 color, FP32 linear view-space depth and a primitive id per pixel.  It
holds none of the synthesis arithmetic, so the CPU oracle and the CUDA path both
take their inputs from here without sharing any method code.

Workloads (shapes, sizes and distributions of the method's VR setting):

* ``small_config``: 256x256, 16 primitives, front depth uniform in 0.3-20 m.
* ``quest_config``: 1832x1920 per eye (the Quest 2 panel quoted in the
  evaluation's real-world apps), 200 primitives plus a ground plane at
  y = -1.6 m, front depth log-uniform in 0.1-100 m.
* ``batch_configs``: 64 frames, 16 each of 1024x1024, 1440x1600, 1832x1920 and
  2064x2208, 50-300 primitives each, IPD uniform in 0.055-0.072 m.
* ``crop_config``: a centred 512x512 crop of the 1832x1920 camera (fx = 916) with the
  quest scene's statistics (the learned inpainter's training frames).

All use a 90 degree horizontal field of view (fx = fy = W/2), the principal point at
the image centre, near 0.05 m and far 1000 m; the source is the left eye at the
origin and the right eye sits at (+IPD, 0, 0).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scene.c")
_LIB_PATH = os.path.join(_HERE, "libyoro_scene.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the ray caster into a shared library beside its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("n_prims", ctypes.c_int32),
                ("ground", ctypes.c_int32), ("log_depth", ctypes.c_int32),
                ("zmin", ctypes.c_float), ("zmax", ctypes.c_float),
                ("rmin", ctypes.c_float), ("rmax", ctypes.c_float),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("far_", ctypes.c_float), ("ground_y", ctypes.c_float),
                ("max_cover", ctypes.c_float)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.scene_render.restype = ctypes.c_int
        lib.scene_render.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_uint64, ctypes.c_float,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        _lib = lib
    return _lib


@dataclasses.dataclass(frozen=True)
class SceneConfig:
    """One synthetic workload: image size, scene statistics and camera."""
    w: int
    h: int
    n_prims: int
    ground: bool
    log_depth: bool
    zmin: float
    zmax: float
    rmin: float = 0.2
    rmax: float = 2.0
    ipd: float = 0.063
    near: float = 0.05
    far: float = 1000.0
    ground_y: float = -1.6
    max_cover: float = 0.25
    focal: float = 0.0  # 0: W/2 (90 degree horizontal FOV); else fx = fy = focal (a centred crop of a wider camera)

    @property
    def fx(self) -> float:
        return self.focal if self.focal > 0 else self.w / 2.0  # 90 degree horizontal FOV: (W/2) / tan(45 deg)

    @property
    def fy(self) -> float:
        return self.fx  # square pixels

    @property
    def cx(self) -> float:
        return self.w / 2.0

    @property
    def cy(self) -> float:
        return self.h / 2.0

    def replace(self, **kw) -> "SceneConfig":
        return dataclasses.replace(self, **kw)

    def camera(self) -> dict:
        """Arguments of ``yoro_create`` for this workload."""
        return dict(w=self.w, h=self.h, fx=self.fx, fy=self.fy, cx=self.cx, cy=self.cy,
                    ipd=self.ipd, near=self.near, far=self.far)


def small_config() -> SceneConfig:
    return SceneConfig(w=256, h=256, n_prims=16, ground=False, log_depth=False, zmin=0.3, zmax=20.0)


def quest_config() -> SceneConfig:
    return SceneConfig(w=1832, h=1920, n_prims=200, ground=True, log_depth=True, zmin=0.1, zmax=100.0)


BATCH_SIZES = ((1024, 1024), (1440, 1600), (1832, 1920), (2064, 2208))


def crop_config(side: int = 512) -> SceneConfig:
    """The centred side x side crop of the 1832x1920 camera (fx = fy = 916, the same
    disparities and hole widths), with the quest scene's statistics: the inpainter's
    training frames."""
    q = quest_config()
    return q.replace(w=side, h=side, focal=q.fx)


def batch_configs(n_frames: int = 64, seed0: int = 1000):
    """Mixed-resolution batch: equal shares of the four per-eye sizes, seeded counts and IPDs.

    Returns a list of (SceneConfig, seed).  Frame i uses seed ``seed0 + i``; its
    primitive count (50-300) and IPD (uniform 0.055-0.072 m) come from a numpy
    Philox stream keyed by that seed.
    """
    out = []
    for i in range(n_frames):
        seed = seed0 + i
        g = np.random.Generator(np.random.Philox(key=seed))
        w, h = BATCH_SIZES[i % len(BATCH_SIZES)]
        n = int(g.integers(50, 301))
        ipd = float(np.float32(g.uniform(0.055, 0.072)))
        out.append((SceneConfig(w=w, h=h, n_prims=n, ground=True, log_depth=True, zmin=0.1,
                                zmax=100.0, ipd=ipd), seed))
    return out


def render(cfg: SceneConfig, seed: int, eye_x: float = 0.0, nthreads: int = 0):
    """Ray-cast one eye: returns (color uint8[H,W,4], depth float32[H,W], prim int32[H,W])."""
    lib = _load()
    c = _Cfg(cfg.w, cfg.h, cfg.n_prims, int(cfg.ground), int(cfg.log_depth), cfg.zmin, cfg.zmax,
             cfg.rmin, cfg.rmax, cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.far, cfg.ground_y,
             cfg.max_cover)
    color = np.empty((cfg.h, cfg.w, 4), np.uint8)
    depth = np.empty((cfg.h, cfg.w), np.float32)
    prim = np.empty((cfg.h, cfg.w), np.int32)
    rc = lib.scene_render(ctypes.byref(c), seed, eye_x, color.ctypes.data, depth.ctypes.data,
                          prim.ctypes.data, nthreads)
    if rc != 0:
        raise RuntimeError("scene_render failed")
    return color, depth, prim


def render_pair(cfg: SceneConfig, seed: int, nthreads: int = 0):
    """Left (source) eye and the analytic right eye of the same scene."""
    return render(cfg, seed, 0.0, nthreads), render(cfg, seed, cfg.ipd, nthreads)
