"""Python binding of the learned hole inpainter's C ABI (``include/yoro_unet.h``).

Argument marshalling only: tensor checks, pointers and streams; every layer runs in
the library's tensor-core kernels (``csrc/unet.cu``).  ``kmajor`` turns a 3x3 weight
array of shape (Cout, Cin, 3, 3) into the K-major layout the kernels read (Cout rows of
9 * Cin values, k = (3 dy + dx) * Cin + ci), padding Cin to a multiple of 32 with zeros.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _check, _stream, load_library

_declared = False


def _lib():
    global _declared
    lib = load_library()
    if not _declared:
        P, I = ctypes.c_void_p, ctypes.c_int
        lib.yoro_unet_conv3x3.argtypes = [P, I, I, I, I, P, P, P, I, I, I, I, I, P]
        lib.yoro_unet_conv3x3.restype = I
        lib.yoro_unet_status.argtypes = [P]
        lib.yoro_unet_status.restype = I
        _declared = True
    return lib


def pad32(c: int) -> int:
    return (c + 31) // 32 * 32


def kmajor(w: np.ndarray) -> np.ndarray:
    """(Cout, Cin, 3, 3) float weights -> (Cout, 9 * pad32(Cin)) float32, k = (3 dy + dx) Cin' + ci."""
    cout, cin = w.shape[:2]
    cp = pad32(cin)
    out = np.zeros((cout, 3, 3, cp), np.float32)
    out[..., :cin] = np.transpose(w, (0, 2, 3, 1))
    return out.reshape(cout, 9 * cp)


def _bf16_ptr(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.bfloat16 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA bfloat16 tensor")
    return t.data_ptr()


def conv3x3(x: torch.Tensor, wk: torch.Tensor, bias: torch.Tensor, y: torch.Tensor, y_coff: int = 0,
            upsample: bool = False, relu: bool = True, stream=None) -> None:
    """yoro_unet_conv3x3: x (T, H, W, Cin) bf16, wk (Cout, 9 Cin) bf16, bias (Cout,) float32,
    y (T, H', W', Cy) bf16 receiving channels y_coff .. y_coff + Cout - 1."""
    T, H, W, Cin = x.shape
    cout = wk.shape[0]
    if wk.shape[1] != 9 * Cin:
        raise ValueError("wk must have 9 * Cin columns")
    if bias.dtype != torch.float32 or not bias.is_cuda or bias.numel() != cout:
        raise ValueError("bias must be a CUDA float32 tensor of Cout values")
    f = 2 if upsample else 1
    if tuple(y.shape[:3]) != (T, f * H, f * W):
        raise ValueError("y has the wrong spatial shape")
    rc = _lib().yoro_unet_conv3x3(_bf16_ptr(x, "x"), T, H, W, Cin, _bf16_ptr(wk, "wk"), bias.data_ptr(),
                                  _bf16_ptr(y, "y"), cout, y.shape[3], int(y_coff), int(bool(upsample)),
                                  int(bool(relu)), _stream(stream))
    _check(rc, "yoro_unet_conv3x3")


def status(stream=None) -> int:
    return _lib().yoro_unet_status(_stream(stream))


class UnetFrame(ctypes.Structure):
    """yoro_unet_frame: one frame of yoro_unet_inpaint_batch."""
    _fields_ = [("w", ctypes.c_int), ("h", ctypes.c_int), ("near_", ctypes.c_float), ("rgba", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("zt", ctypes.c_void_p), ("src_depth", ctypes.c_void_p)]


def _check_frame_tensors(rgba, mask, zt, src_depth):
    h, w = mask.shape
    for t, dt, shp, name in ((rgba, torch.uint8, (h, w, 4), "rgba"), (mask, torch.uint8, (h, w), "mask"),
                             (zt, torch.float32, (h, w), "zt"), (src_depth, torch.float32, (h, w), "src_depth")):
        if not t.is_cuda or t.dtype != dt or tuple(t.shape) != shp or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor {shp}")
    return w, h


def _lib_net():
    lib = _lib()
    if not hasattr(lib, "_net_declared"):
        P, I, F, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong
        lib.yoro_unet_param_count.argtypes = []
        lib.yoro_unet_param_count.restype = L
        lib.yoro_unet_create.argtypes = [P, L, I, I, I]
        lib.yoro_unet_create.restype = P
        lib.yoro_unet_destroy.argtypes = [P]
        lib.yoro_unet_destroy.restype = None
        lib.yoro_unet_forward.argtypes = [P, P, I, P, P]
        lib.yoro_unet_forward.restype = I
        lib.yoro_unet_inpaint.argtypes = [P, I, I, F, P, P, P, P, P]
        lib.yoro_unet_inpaint.restype = I
        lib.yoro_unet_prepare.argtypes = [P, I, I, F, P, P, P, P, P, I, P, P, P]
        lib.yoro_unet_prepare.restype = I
        lib.yoro_unet_inpaint_batch.argtypes = [P, I, ctypes.POINTER(UnetFrame), P]
        lib.yoro_unet_inpaint_batch.restype = I
        lib._net_declared = True
    return lib


def param_count() -> int:
    return int(_lib_net().yoro_unet_param_count())


def flatten_params(p: dict, names) -> np.ndarray:
    """Parameters as one float32 array in the order of ``names`` (the definition's layer
    order): each layer's weights, then its biases."""
    parts = []
    for name in names:
        parts += [np.asarray(p[name + ".w"], np.float32).reshape(-1), np.asarray(p[name + ".b"], np.float32)]
    return np.concatenate(parts)


class Inpainter:
    """yoro_unet_create / destroy, forward and inpaint."""

    def __init__(self, params: np.ndarray, max_tiles: int = 0, max_w: int = 0, max_h: int = 0):
        params = np.ascontiguousarray(params, np.float32)
        lib = _lib_net()
        self.ptr = lib.yoro_unet_create(params.ctypes.data, params.size, int(max_tiles), int(max_w), int(max_h))
        if not self.ptr:
            raise RuntimeError("yoro_unet_create failed (parameter count or allocation)")

    def forward(self, x: torch.Tensor, rgb: torch.Tensor, stream=None) -> None:
        """x (T, 64, 64, 32) bf16 -> rgb (T, 64, 64, 3) float32."""
        T = x.shape[0]
        if tuple(x.shape[1:]) != (64, 64, 32):
            raise ValueError("x must be (T, 64, 64, 32)")
        if rgb.dtype != torch.float32 or tuple(rgb.shape) != (T, 64, 64, 3) or not rgb.is_cuda:
            raise ValueError("rgb must be a CUDA float32 tensor (T, 64, 64, 3)")
        _check(_lib_net().yoro_unet_forward(self.ptr, _bf16_ptr(x, "x"), T, rgb.data_ptr(), _stream(stream)),
               "yoro_unet_forward")

    def inpaint(self, rgba: torch.Tensor, mask: torch.Tensor, zt: torch.Tensor, src_depth: torch.Tensor,
                near: float, stream=None) -> None:
        """In place: hole pixels of rgba (h, w, 4) uint8 take the network's colors."""
        w, h = _check_frame_tensors(rgba, mask, zt, src_depth)
        _check(_lib_net().yoro_unet_inpaint(self.ptr, w, h, float(near), rgba.data_ptr(), mask.data_ptr(),
                                            zt.data_ptr(), src_depth.data_ptr(), _stream(stream)),
               "yoro_unet_inpaint")

    def inpaint_batch(self, frames, stream=None) -> None:
        """yoro_unet_inpaint_batch: frames = [(rgba, mask, zt, src_depth, near), ...], each
        repainted in place as inpaint() would, in as few passes of the network as fit."""
        arr = (UnetFrame * max(1, len(frames)))()
        for i, (rgba, mask, zt, src_depth, near) in enumerate(frames):
            w, h = _check_frame_tensors(rgba, mask, zt, src_depth)
            arr[i] = UnetFrame(w, h, float(near), rgba.data_ptr(), mask.data_ptr(), zt.data_ptr(),
                               src_depth.data_ptr())
        _check(_lib_net().yoro_unet_inpaint_batch(self.ptr, len(frames), arr, _stream(stream)),
               "yoro_unet_inpaint_batch")

    def prepare(self, rgba, mask, zt, src_depth, near: float, x_out: torch.Tensor, stream=None) -> np.ndarray:
        """The network inputs of the frame's hole tiles into x_out[:count]; returns the tile
        indices (ty * ceil(w / 64) + tx)."""
        h, w = mask.shape
        ntiles = ((w + 63) // 64) * ((h + 63) // 64)
        if x_out.shape[0] < ntiles or tuple(x_out.shape[1:]) != (64, 64, 32):
            raise ValueError("x_out must hold (>= tiles of the frame, 64, 64, 32)")
        lst = np.zeros(ntiles, np.int32)
        cnt = np.zeros(1, np.int32)
        _check(_lib_net().yoro_unet_prepare(self.ptr, w, h, float(near), rgba.data_ptr(), mask.data_ptr(),
                                            zt.data_ptr(), src_depth.data_ptr(), _bf16_ptr(x_out, "x_out"), ntiles,
                                            lst.ctypes.data, cnt.ctypes.data, _stream(stream)), "yoro_unet_prepare")
        return lst[:int(cnt[0])].copy()

    def close(self) -> None:
        if self.ptr:
            _lib_net().yoro_unet_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def _lib_train():
    lib = _lib_net()
    if not hasattr(lib, "_train_declared"):
        P, I, F, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong
        lib.yoro_unet_trainer_create.argtypes = [P, L, I, F, F, F, F]
        lib.yoro_unet_trainer_create.restype = P
        lib.yoro_unet_trainer_destroy.argtypes = [P]
        lib.yoro_unet_trainer_destroy.restype = None
        lib.yoro_unet_train_step.argtypes = [P, P, P, P, I, P]
        lib.yoro_unet_train_step.restype = I
        lib.yoro_unet_trainer_read.argtypes = [P, I, P, P]
        lib.yoro_unet_trainer_read.restype = I
        lib.yoro_unet_trainer_set_lr.argtypes = [P, F]
        lib.yoro_unet_trainer_set_lr.restype = I
        lib._train_declared = True
    return lib


class Trainer:
    """yoro_unet_trainer_*: Adam on the GPU from an initial parameter array."""

    def __init__(self, params: np.ndarray, batch_tiles: int, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        params = np.ascontiguousarray(params, np.float32)
        self.n = params.size
        self.ptr = _lib_train().yoro_unet_trainer_create(params.ctypes.data, params.size, int(batch_tiles), lr, beta1,
                                                         beta2, eps)
        if not self.ptr:
            raise RuntimeError("yoro_unet_trainer_create failed")

    def step(self, x: torch.Tensor, gt: torch.Tensor, hole: torch.Tensor, stream=None) -> None:
        T = x.shape[0]
        if tuple(x.shape) != (T, 64, 64, 32):
            raise ValueError("x must be (T, 64, 64, 32) bf16")
        for t, shp, name in ((gt, (T, 64, 64, 3), "gt"), (hole, (T, 64, 64), "hole")):
            if not t.is_cuda or t.dtype != torch.uint8 or tuple(t.shape) != shp or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA uint8 tensor {shp}")
        _check(_lib_train().yoro_unet_train_step(self.ptr, _bf16_ptr(x, "x"), gt.data_ptr(), hole.data_ptr(), T,
                                                 _stream(stream)), "yoro_unet_train_step")

    def set_lr(self, lr: float) -> None:
        _check(_lib_train().yoro_unet_trainer_set_lr(self.ptr, float(lr)), "yoro_unet_trainer_set_lr")

    def read(self, what: str, stream=None) -> np.ndarray:
        code = {"params": 0, "grads": 1, "loss": 2}[what]
        out = np.empty(1 if code == 2 else self.n, np.float32)
        _check(_lib_train().yoro_unet_trainer_read(self.ptr, code, out.ctypes.data, _stream(stream)),
               "yoro_unet_trainer_read")
        return out

    def close(self) -> None:
        if self.ptr:
            _lib_train().yoro_unet_trainer_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass
