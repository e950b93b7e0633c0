"""GB300 second-eye synthesis (YORO): Python binding of ``libyoro.so``.

The functions below carry the names of the C ABI in ``include/yoro.h`` and only
marshal arguments (tensor checks, pointers, streams); every step of the path runs
in the library's CUDA kernels.  PyTorch supplies device memory and streams.  The
library is loaded from ``paper_2506_15183_gb300/_lib/libyoro.so``; if it has not
been built, every call raises ``RuntimeError`` (there is no CPU fallback).  A process
that calls ``load_library(debug=True)`` before any other call uses the debug-bounds
build ``libyoro_debug.so`` instead (``_build.build_cuda(debug=True)`` makes it).
"""
from __future__ import annotations

import ctypes
import os

import torch

__all__ = [
    "YoroError", "Synthesizer", "load_library", "yoro_create", "yoro_destroy", "yoro_synthesize",
    "yoro_synthesize_unfused", "yoro_synthesize_host", "yoro_synthesize_batch", "yoro_stream_status",
    "yoro_max_fused_width", "yoro_status_string", "yoro_last_create_error", "STATUS",
    "yoro_synthesize_noalloc", "yoro_noalloc_max_pixels", "yoro_tune_batch", "yoro_batch_band",
    "yoro_reset_tuning", "yoro_create_ex", "yoro_synthesize_mapped", "yoro_debug_bounds_enabled",
    "yoro_debug_selftest", "yoro_create_imb", "yoro_create_pose", "yoro_synthesize_zt",
]

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libyoro.so")
_DEBUG_LIB_PATH = os.path.join(os.path.dirname(_LIB_PATH), "libyoro_debug.so")
_lib = None

STATUS = {0: "YORO_OK", 1: "YORO_EINVAL", 2: "YORO_EALIGN", 3: "YORO_ENOMEM", 4: "YORO_ECUDA",
          5: "YORO_EDEVICE", 6: "YORO_ETOOBIG", 7: "YORO_ETIMEOUT", 8: "YORO_ECANCELED"}


class YoroError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_status_string(code)})")


class _Options(ctypes.Structure):
    _fields_ = [("kernel_rows", ctypes.c_int), ("nearest_first", ctypes.c_int)]


class _Frame(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int), ("h", ctypes.c_int),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("ipd", ctypes.c_float), ("near_", ctypes.c_float),
                ("far_", ctypes.c_float),
                ("color", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("out_color", ctypes.c_void_p), ("out_hole_mask", ctypes.c_void_p)]


def load_library(path: str | None = None, debug: bool = False) -> ctypes.CDLL:
    """Load libyoro.so (built by ``__graft_entry__.build()``), or with ``debug`` the
    debug-bounds build; raise if it is missing.  The first call decides for the process."""
    global _lib
    if _lib is not None:
        if debug and not _lib.yoro_debug_bounds_enabled():
            raise RuntimeError("the release library is already loaded in this process")
        return _lib
    path = path or (_DEBUG_LIB_PATH if debug else _LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError(f"libyoro.so not built ({path}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    lib.yoro_create.argtypes = [I, I, F, F, F, F, F, F, F]
    lib.yoro_create.restype = P
    lib.yoro_create_ex.argtypes = [I, I, F, F, F, F, F, F, F, ctypes.POINTER(_Options)]
    lib.yoro_create_ex.restype = P
    lib.yoro_create_imb.argtypes = [I, I, F, F, F, F, F, F, F, ctypes.POINTER(_Options), I, I]
    lib.yoro_create_imb.restype = P
    lib.yoro_create_pose.argtypes = [I, I, F, F, F, F, P, P, F, F, ctypes.POINTER(_Options)]
    lib.yoro_create_pose.restype = P
    lib.yoro_last_create_error.argtypes = []
    lib.yoro_last_create_error.restype = I
    lib.yoro_destroy.argtypes = [P]
    lib.yoro_destroy.restype = None
    for name in ("yoro_synthesize", "yoro_synthesize_unfused", "yoro_synthesize_host", "yoro_synthesize_mapped"):
        fn = getattr(lib, name)
        fn.argtypes = [P, P, P, P, P, P]
        fn.restype = I
    lib.yoro_synthesize_batch.argtypes = [I, ctypes.POINTER(_Frame), P]
    lib.yoro_synthesize_batch.restype = I
    lib.yoro_stream_status.argtypes = [P, P]
    lib.yoro_stream_status.restype = I
    lib.yoro_max_fused_width.argtypes = []
    lib.yoro_max_fused_width.restype = I
    lib.yoro_status_string.argtypes = [I]
    lib.yoro_status_string.restype = ctypes.c_char_p
    lib.yoro_synthesize_noalloc.argtypes = [I, I, F, F, F, F, F, F, F, P, P, P, P, P]
    lib.yoro_synthesize_noalloc.restype = I
    lib.yoro_noalloc_max_pixels.argtypes = []
    lib.yoro_noalloc_max_pixels.restype = I
    lib.yoro_tune_batch.argtypes = [I, ctypes.POINTER(_Frame), I, P, ctypes.POINTER(I)]
    lib.yoro_tune_batch.restype = I
    lib.yoro_batch_band.argtypes = [I]
    lib.yoro_batch_band.restype = I
    lib.yoro_reset_tuning.argtypes = []
    lib.yoro_reset_tuning.restype = None
    lib.yoro_debug_bounds_enabled.argtypes = []
    lib.yoro_debug_bounds_enabled.restype = I
    lib.yoro_debug_selftest.argtypes = [P]
    lib.yoro_debug_selftest.restype = I
    lib.yoro_synthesize_zt.argtypes = [P, P, P, P, P, P, P]
    lib.yoro_synthesize_zt.restype = I
    _lib = lib
    return lib


def _status_string(code: int) -> str:
    try:
        return load_library().yoro_status_string(code).decode()
    except Exception:  # noqa: BLE001 - message only
        return "?"


def _check(code: int, where: str) -> None:
    if code != 0:
        raise YoroError(code, where)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev_ptr(t: torch.Tensor, dtype, shape, name: str) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)}")
    return t.data_ptr()


def _host_ptr(t: torch.Tensor, dtype, shape, name: str) -> int:
    if t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}")
    return t.data_ptr()


class _Handle:
    """A yoro_handle plus the frame size it was created for."""

    def __init__(self, ptr: int, w: int, h: int):
        self.ptr, self.w, self.h = ptr, w, h


def yoro_last_create_error() -> int:
    return load_library().yoro_last_create_error()


def yoro_create(w, h, fx, fy, cx, cy, ipd, near, far) -> _Handle:
    lib = load_library()
    p = lib.yoro_create(int(w), int(h), fx, fy, cx, cy, ipd, near, far)
    if not p:
        raise YoroError(lib.yoro_last_create_error(), "yoro_create")
    return _Handle(p, int(w), int(h))


def yoro_create_ex(w, h, fx, fy, cx, cy, ipd, near, far, kernel_rows=3, nearest_first=False) -> _Handle:
    """yoro_create with a Patcher kernel variant (height kernel_rows, nearest-first order)."""
    lib = load_library()
    opt = _Options(int(kernel_rows), int(bool(nearest_first)))
    p = lib.yoro_create_ex(int(w), int(h), fx, fy, cx, cy, ipd, near, far, ctypes.byref(opt))
    if not p:
        raise YoroError(lib.yoro_last_create_error(), "yoro_create_ex")
    return _Handle(p, int(w), int(h))


def yoro_create_imb(w, h, fx, fy, cx, cy, ipd, near, far, kernel_rows=3, nearest_first=False, imbuffer_div=1,
                    interpolate=False) -> _Handle:
    """yoro_create_ex through the row-downsampled intermediate buffer: cells of
    imbuffer_div pixels (1, 2, 4, 8, 16) and, with interpolate, the shift interpolated
    between cells and the source sampled linearly."""
    lib = load_library()
    opt = _Options(int(kernel_rows), int(bool(nearest_first)))
    p = lib.yoro_create_imb(int(w), int(h), fx, fy, cx, cy, ipd, near, far, ctypes.byref(opt), int(imbuffer_div),
                            int(bool(interpolate)))
    if not p:
        raise YoroError(lib.yoro_last_create_error(), "yoro_create_imb")
    return _Handle(p, int(w), int(h))


def yoro_create_pose(w, h, fx, fy, cx, cy, rotation, position, near, far, kernel_rows=3,
                     nearest_first=False) -> _Handle:
    """A context for a general second-eye pose: rotation (3x3, row-major) and position
    (3) of the second eye in left-eye camera coordinates, p' = rotation (p - position)."""
    lib = load_library()
    rot = (ctypes.c_float * 9)(*[float(v) for v in _flat(rotation, 9, "rotation")])
    pos = (ctypes.c_float * 3)(*[float(v) for v in _flat(position, 3, "position")])
    opt = _Options(int(kernel_rows), int(bool(nearest_first)))
    p = lib.yoro_create_pose(int(w), int(h), fx, fy, cx, cy, rot, pos, near, far, ctypes.byref(opt))
    if not p:
        raise YoroError(lib.yoro_last_create_error(), "yoro_create_pose")
    return _Handle(p, int(w), int(h))


def _flat(a, n, name):
    vals = [v for row in a for v in (row if hasattr(row, "__len__") else [row])]
    if len(vals) != n:
        raise ValueError(f"{name} must have {n} values")
    return vals


def yoro_destroy(h: _Handle) -> None:
    if h is not None and h.ptr:
        load_library().yoro_destroy(h.ptr)
        h.ptr = None


def _frame_ptrs(h: _Handle, color, depth, out_color, out_mask, ptr):
    return (ptr(color, torch.uint8, (h.h, h.w, 4), "color"), ptr(depth, torch.float32, (h.h, h.w), "depth"),
            ptr(out_color, torch.uint8, (h.h, h.w, 4), "out_color"),
            ptr(out_mask, torch.uint8, (h.h, h.w), "out_hole_mask"))


def yoro_synthesize(h: _Handle, color, depth, out_color, out_mask, stream=None) -> None:
    """Right eye of one frame into out_color/out_mask (device tensors), on `stream`."""
    p = _frame_ptrs(h, color, depth, out_color, out_mask, _dev_ptr)
    _check(load_library().yoro_synthesize(h.ptr, *p, _stream(stream)), "yoro_synthesize")


def yoro_synthesize_zt(h: _Handle, color, depth, out_color, out_mask, out_zt, stream=None) -> None:
    """yoro_synthesize that also writes the warped depth (0 at holes) into out_zt (h, w) float32."""
    p = _frame_ptrs(h, color, depth, out_color, out_mask, _dev_ptr)
    z = _dev_ptr(out_zt, torch.float32, (h.h, h.w), "out_zt")
    _check(load_library().yoro_synthesize_zt(h.ptr, *p, z, _stream(stream)), "yoro_synthesize_zt")


def yoro_synthesize_unfused(h: _Handle, color, depth, out_color, out_mask, stream=None) -> None:
    p = _frame_ptrs(h, color, depth, out_color, out_mask, _dev_ptr)
    _check(load_library().yoro_synthesize_unfused(h.ptr, *p, _stream(stream)), "yoro_synthesize_unfused")


def yoro_synthesize_host(h: _Handle, color, depth, out_color, out_mask, stream=None) -> None:
    """Host tensors in and out (pinned for asynchronous copies); synchronise before reading."""
    p = _frame_ptrs(h, color, depth, out_color, out_mask, _host_ptr)
    _check(load_library().yoro_synthesize_host(h.ptr, *p, _stream(stream)), "yoro_synthesize_host")


def _frame_array(frames):
    arr = (_Frame * max(len(frames), 1))()
    for i, fr in enumerate(frames):
        w, hh = int(fr["w"]), int(fr["h"])
        arr[i] = _Frame(w, hh, fr["fx"], fr["fy"], fr["cx"], fr["cy"], fr["ipd"], fr["near"], fr["far"],
                        _dev_ptr(fr["color"], torch.uint8, (hh, w, 4), "color"),
                        _dev_ptr(fr["depth"], torch.float32, (hh, w), "depth"),
                        _dev_ptr(fr["out_color"], torch.uint8, (hh, w, 4), "out_color"),
                        _dev_ptr(fr["out_mask"], torch.uint8, (hh, w), "out_hole_mask"))
    return arr


def yoro_synthesize_mapped(h: _Handle, color, depth, out_color, out_mask, stream=None) -> None:
    """Host tensors in page-locked memory (``pin_memory()``), read and written by the kernel
    directly (zero copy); synchronise before reading."""
    p = _frame_ptrs(h, color, depth, out_color, out_mask, _host_ptr)
    _check(load_library().yoro_synthesize_mapped(h.ptr, *p, _stream(stream)), "yoro_synthesize_mapped")


def yoro_synthesize_batch(frames, stream=None) -> None:
    """frames: sequence of dicts with keys w, h, fx, fy, cx, cy, ipd, near, far, color, depth,
    out_color, out_mask (device tensors)."""
    arr = _frame_array(frames)
    _check(load_library().yoro_synthesize_batch(len(frames), arr, _stream(stream)), "yoro_synthesize_batch")


def yoro_tune_batch(frames, reps: int = 3, stream=None) -> int:
    """Time the batch at several band heights, keep the fastest for later batch launches of
    the same widest width on this device, and return it (synchronises the stream)."""
    arr = _frame_array(frames)
    band = ctypes.c_int(0)
    _check(load_library().yoro_tune_batch(len(frames), arr, int(reps), _stream(stream), ctypes.byref(band)),
           "yoro_tune_batch")
    return band.value


def yoro_batch_band(w: int) -> int:
    return load_library().yoro_batch_band(int(w))


def yoro_reset_tuning() -> None:
    load_library().yoro_reset_tuning()


def yoro_synthesize_noalloc(w, h, fx, fy, cx, cy, ipd, near, far, color, depth, out_color, out_mask,
                            stream=None) -> None:
    """Right eye without a handle and without device allocation (for callers that must not
    allocate where they synthesize); frames up to yoro_noalloc_max_pixels() pixels.  Calls
    share one scratch array in the library, so they must not overlap on the GPU."""
    w, h = int(w), int(h)
    p = (_dev_ptr(color, torch.uint8, (h, w, 4), "color"), _dev_ptr(depth, torch.float32, (h, w), "depth"),
         _dev_ptr(out_color, torch.uint8, (h, w, 4), "out_color"),
         _dev_ptr(out_mask, torch.uint8, (h, w), "out_hole_mask"))
    _check(load_library().yoro_synthesize_noalloc(w, h, fx, fy, cx, cy, ipd, near, far, *p, _stream(stream)),
           "yoro_synthesize_noalloc")


def yoro_noalloc_max_pixels() -> int:
    return load_library().yoro_noalloc_max_pixels()


def yoro_stream_status(h: _Handle | None, stream=None) -> int:
    return load_library().yoro_stream_status(h.ptr if h is not None else None, _stream(stream))


def yoro_max_fused_width() -> int:
    return load_library().yoro_max_fused_width()


def yoro_debug_bounds_enabled() -> bool:
    return bool(load_library().yoro_debug_bounds_enabled())


def yoro_debug_selftest(stream=None) -> None:
    _check(load_library().yoro_debug_selftest(_stream(stream)), "yoro_debug_selftest")


def yoro_status_string(code: int) -> str:
    return _status_string(code)


class Synthesizer:
    """Owns a handle for one camera; ``__call__`` allocates the outputs with torch."""

    def __init__(self, w, h, fx, fy, cx, cy, ipd, near=0.05, far=1000.0, kernel_rows=3, nearest_first=False,
                 imbuffer_div=1, interpolate=False, pose=None):
        """pose: None (the stereo pair at +ipd along x) or (rotation 3x3, position 3) of a
        general second eye, which then replaces ipd."""
        self.w, self.h = int(w), int(h)
        if pose is not None:
            self.handle = yoro_create_pose(w, h, fx, fy, cx, cy, pose[0], pose[1], near, far, kernel_rows,
                                           nearest_first)
        elif imbuffer_div != 1 or interpolate:
            self.handle = yoro_create_imb(w, h, fx, fy, cx, cy, ipd, near, far, kernel_rows, nearest_first,
                                          imbuffer_div, interpolate)
        elif kernel_rows == 3 and not nearest_first:
            self.handle = yoro_create(w, h, fx, fy, cx, cy, ipd, near, far)
        else:
            self.handle = yoro_create_ex(w, h, fx, fy, cx, cy, ipd, near, far, kernel_rows, nearest_first)

    def __call__(self, color: torch.Tensor, depth: torch.Tensor, stream=None, unfused: bool = False):
        out = torch.empty((self.h, self.w, 4), dtype=torch.uint8, device=color.device)
        mask = torch.empty((self.h, self.w), dtype=torch.uint8, device=color.device)
        fn = yoro_synthesize_unfused if unfused else yoro_synthesize
        fn(self.handle, color, depth, out, mask, stream)
        return out, mask

    def status(self, stream=None) -> int:
        return yoro_stream_status(self.handle, stream)

    def close(self) -> None:
        yoro_destroy(self.handle)

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass
