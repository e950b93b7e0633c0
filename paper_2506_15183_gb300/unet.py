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
