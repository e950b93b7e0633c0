"""Plain CPU definition of the learned hole inpainter (a U-Net over hole-containing tiles).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: it defines what a GPU inpainter
must compute, slowly and literally, and shares nothing with the CUDA library.

The paper's Patcher is the hand-written fill of Alg. 3 and Eq. 6; a learned inpainter
is an extension of the method (its comparison system is a GAN, not reproduced).  The
network defined here is a 4-level U-Net:

  input    6 channels per pixel of a tile: the plain path's right eye (3, in [0, 1]:
           the warped color, and at holes the Patcher's fill, which the network refines),
           the hole mask (1 at holes), the warped depth and the source-eye depth at the
           same pixel (each as near / depth, in (0, 1]; the warped depth zero at holes)
  encoder  level l (l = 0..3, widths 32, 64, 128, 256): two 3x3 convolutions with zero
           padding, each followed by ReLU; between levels a 2x2 max pool
  decoder  level l (l = 2..0): nearest 2x upsampling of level l + 1, concatenated after
           the encoder's level-l output (skip first), two 3x3 convolutions with ReLU
  output   a 1x1 convolution to 3 channels and a logistic sigmoid: the color in [0, 1]
  compose  hole pixels take the network's color (times 255, rounded half to even),
           reached pixels keep the warped color

Precision: weights and activations are BF16, accumulation FP32.  Here: every weight and
every input element is rounded to bfloat16 (round to nearest even) before use; each
convolution sums the products of BF16 values in FP32 (the products are exact in FP32)
in the order input channel, then kernel row, then kernel column; the bias is added in
FP32; the ReLU output is rounded to BF16 and is the next layer's input.  The order of a
GPU's tensor-core accumulation is not this order, so a kernel is compared with this
definition within a tolerance derived from the FP32 sums, not bit for bit.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (32, 64, 128, 256)
IN_CH = 6
OUT_CH = 3


def bf16(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32.
    NaN stays NaN; infinities stay infinite."""
    shape = np.shape(x)
    a = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).copy()
    nan = np.isnan(a)
    out[nan] = a[nan]
    return out.reshape(shape)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """3x3 convolution with zero padding: x (C, H, W), w (K, C, 3, 3), b (K,) -> (K, H, W).

    FP32 sums of BF16 products in the order input channel, kernel row, kernel column
    (for each output element), then the bias."""
    c, h, wd = x.shape
    k = w.shape[0]
    xp = np.zeros((c, h + 2, wd + 2), np.float32)
    xp[:, 1:-1, 1:-1] = x
    acc = np.zeros((k, h, wd), np.float32)
    for ci in range(c):
        for dy in range(3):
            for dx in range(3):
                # one product per output element, added in the stated order
                acc = acc + w[:, ci, dy, dx][:, None, None] * xp[ci, dy:dy + h, dx:dx + wd][None, :, :]
    return acc + b[:, None, None]


def conv1x1(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """1x1 convolution: x (C, H, W), w (K, C), b (K,); sums in input-channel order."""
    acc = np.zeros((w.shape[0],) + x.shape[1:], np.float32)
    for ci in range(x.shape[0]):
        acc = acc + w[:, ci][:, None, None] * x[ci][None, :, :]
    return acc + b[:, None, None]


def relu_bf16(x: np.ndarray) -> np.ndarray:
    return bf16(np.maximum(x, np.float32(0.0)))


def maxpool2(x: np.ndarray) -> np.ndarray:
    c, h, w = x.shape
    return x[:, : h // 2 * 2, : w // 2 * 2].reshape(c, h // 2, 2, w // 2, 2).max(axis=(2, 4))


def upsample2(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def layer_shapes():
    """(name, weight shape, bias shape) of every layer, in the order the weights are stored."""
    shapes = []
    cin = IN_CH
    for l, c in enumerate(WIDTHS):
        shapes += [(f"enc{l}a", (c, cin, 3, 3), (c,)), (f"enc{l}b", (c, c, 3, 3), (c,))]
        cin = c
    for l in range(len(WIDTHS) - 2, -1, -1):
        c = WIDTHS[l]
        shapes += [(f"dec{l}a", (c, c + WIDTHS[l + 1], 3, 3), (c,)), (f"dec{l}b", (c, c, 3, 3), (c,))]
    shapes.append(("out", (OUT_CH, WIDTHS[0]), (OUT_CH,)))
    return shapes


def init_weights(seed: int) -> dict:
    """He-normal weights (BF16-rounded) and zero biases, seeded."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ws, bs in layer_shapes():
        fan_in = int(np.prod(ws[1:]))
        p[name + ".w"] = bf16(rng.normal(0.0, np.sqrt(2.0 / fan_in), ws).astype(np.float32))
        p[name + ".b"] = np.zeros(bs, np.float32)
    return p


def forward(x: np.ndarray, p: dict) -> np.ndarray:
    """The network on one tile: x (6, H, W) with H, W multiples of 8 -> color (3, H, W) in [0, 1]."""
    assert x.shape[0] == IN_CH and x.shape[1] % 8 == 0 and x.shape[2] % 8 == 0
    p = {k: (bf16(v) if k.endswith(".w") else np.asarray(v, np.float32)) for k, v in p.items()}
    a = bf16(x)
    skips = []
    for l in range(len(WIDTHS)):
        if l:
            a = maxpool2(a)
        a = relu_bf16(conv3x3(a, p[f"enc{l}a.w"], p[f"enc{l}a.b"]))
        a = relu_bf16(conv3x3(a, p[f"enc{l}b.w"], p[f"enc{l}b.b"]))
        skips.append(a)
    for l in range(len(WIDTHS) - 2, -1, -1):
        a = np.concatenate([skips[l], upsample2(a)], axis=0)
        a = relu_bf16(conv3x3(a, p[f"dec{l}a.w"], p[f"dec{l}a.b"]))
        a = relu_bf16(conv3x3(a, p[f"dec{l}b.w"], p[f"dec{l}b.b"]))
    z = conv1x1(a, p["out.w"], p["out.b"])
    return (np.float32(1.0) / (np.float32(1.0) + np.exp(-z, dtype=np.float32))).astype(np.float32)


def tile_input(color: np.ndarray, mask: np.ndarray, zt: np.ndarray, zsrc: np.ndarray, near: float) -> np.ndarray:
    """The 6 input channels of a tile from the plain path's right eye (H, W, 4 uint8: the
    reached pixels' warped colors and the Patcher's fill at the holes), its hole mask
    (H, W), warped depth zt (H, W; ignored at holes) and the source eye's depth (H, W):
    color / 255 everywhere, the mask, and near / depth (zero at holes for the warped
    depth)."""
    hole = mask.astype(bool)
    x = np.zeros((IN_CH,) + mask.shape, np.float32)
    x[0:3] = color[..., :3].transpose(2, 0, 1).astype(np.float32) / np.float32(255.0)
    x[3] = hole.astype(np.float32)
    x[4] = np.where(hole, 0.0, np.float32(near) / np.maximum(zt, np.float32(near)))
    x[5] = np.float32(near) / np.maximum(zsrc, np.float32(near))
    return x


def compose(warped: np.ndarray, mask: np.ndarray, color: np.ndarray) -> np.ndarray:
    """Hole pixels take the network's color (x 255, rounded half to even, alpha 255);
    reached pixels keep the warped color."""
    out = warped.copy()
    hole = mask.astype(bool)
    net = np.rint(np.clip(color, 0.0, 1.0) * np.float32(255.0)).astype(np.uint8).transpose(1, 2, 0)
    out[..., :3][hole] = net[hole]
    out[..., 3][hole] = 255
    return out


# ---- training: the loss and its gradient (test infrastructure for the GPU trainer) ----
#
# Loss of one batch: the mean over hole pixels and color channels of the squared error
# between the network's color and the ground truth (in [0, 1]):
#     L = sum_{hole pixels, c} (s_c - g_c)^2 / (3 * number of hole pixels).
# The gradient is the chain rule through the network written out layer by layer (no
# automatic differentiation): sigmoid' = s (1 - s); the 1x1 layer's transpose; ReLU'
# = 1 where the layer's output is positive; a 3x3 convolution's data gradient is the
# full correlation of the output gradient with the kernel flipped in both directions and
# transposed in its channels, its weight gradient the correlation of the input with the
# output gradient; 2x2 max pooling sends the gradient to the first maximum of its window
# (row-major order); nearest upsampling sums the four gradients of a 2x2 block; a
# concatenation splits the gradient by channels.  With exact=True every array is float64
# and nothing is rounded to bfloat16 (the form the finite-difference pin checks); with
# exact=False the forward is the definition's (bfloat16 activations), and the backward
# runs in float64 through those activations.

def _conv3x3_64(x, w, b):
    c, h, wd = x.shape
    xp = np.zeros((c, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[0], h, wd))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("kc,chw->khw", w[:, :, dy, dx], xp[:, dy:dy + h, dx:dx + wd])
    return out + b[:, None, None]


def _conv3x3_backward(x, w, dz):
    """(dx, dw, db) of y = conv3x3(x, w) + b given dz = dL/dy (float64)."""
    c, h, wd = x.shape
    xp = np.zeros((c, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    dw = np.zeros(w.shape)
    dxp = np.zeros((c, h + 2, wd + 2))
    for dy in range(3):
        for dx in range(3):
            dw[:, :, dy, dx] = np.einsum("khw,chw->kc", dz, xp[:, dy:dy + h, dx:dx + wd])
            dxp[:, dy:dy + h, dx:dx + wd] += np.einsum("kc,khw->chw", w[:, :, dy, dx], dz)
    return dxp[:, 1:-1, 1:-1], dw, dz.sum(axis=(1, 2))


def _maxpool_backward(x, dy):
    """Gradient of 2x2 max pooling: each window's gradient to its first maximum (row-major)."""
    c, h, w = x.shape
    win = x.reshape(c, h // 2, 2, w // 2, 2).transpose(0, 1, 3, 2, 4).reshape(c, h // 2, w // 2, 4)
    first = np.argmax(win == win.max(axis=-1, keepdims=True), axis=-1)
    dx = np.zeros((c, h // 2, w // 2, 4))
    np.put_along_axis(dx, first[..., None], dy[..., None], axis=-1)
    return dx.reshape(c, h // 2, w // 2, 2, 2).transpose(0, 1, 3, 2, 4).reshape(c, h, w)


def loss_and_grads(x: np.ndarray, p: dict, gt: np.ndarray, hole: np.ndarray, exact: bool = False):
    """Loss (float) and gradients {name.w, name.b} (float64) of the network on tile x (6, H,
    W), ground truth gt (3, H, W) in [0, 1] and hole mask (H, W)."""
    f = (lambda a: np.asarray(a, np.float64)) if exact else (lambda a: bf16(a).astype(np.float64))
    P = {k: (f(v) if k.endswith(".w") else np.asarray(v, np.float64)) for k, v in p.items()}
    conv = _conv3x3_64 if exact else (lambda a, w, b: conv3x3(a.astype(np.float32), w.astype(np.float32),
                                                             b.astype(np.float32)).astype(np.float64))
    act = (lambda z: np.maximum(z, 0.0)) if exact else (lambda z: bf16(np.maximum(z, 0.0).astype(np.float32))
                                                         .astype(np.float64))
    a = f(x)
    saved, skips = [], []
    for l in range(len(WIDTHS)):
        if l:
            pooled_from = a
            a = a.reshape(a.shape[0], a.shape[1] // 2, 2, a.shape[2] // 2, 2).max(axis=(2, 4))
            saved.append(("pool", l, pooled_from))
        for s in "ab":
            y = act(conv(a, P[f"enc{l}{s}.w"], P[f"enc{l}{s}.b"]))
            saved.append(("conv", f"enc{l}{s}", a, y))
            a = y
        skips.append(a)
    for l in range(len(WIDTHS) - 2, -1, -1):
        up = np.repeat(np.repeat(a, 2, axis=1), 2, axis=2)
        saved.append(("cat", l, skips[l].shape[0]))
        a = np.concatenate([skips[l], up], axis=0)
        for s in "ab":
            y = act(conv(a, P[f"dec{l}{s}.w"], P[f"dec{l}{s}.b"]))
            saved.append(("conv", f"dec{l}{s}", a, y))
            a = y
    wo, bo = P["out.w"], P["out.b"]
    z = np.einsum("kc,chw->khw", wo, a) + bo[:, None, None]
    s_ = 1.0 / (1.0 + np.exp(-z))
    m = hole.astype(bool)[None]
    n = 3 * int(hole.astype(bool).sum())
    err = np.where(m, s_ - gt, 0.0)
    loss = float((err ** 2).sum() / n)
    dzo = 2.0 * err / n * s_ * (1.0 - s_)
    g = {"out.w": np.einsum("khw,chw->kc", dzo, a), "out.b": dzo.sum(axis=(1, 2))}
    da = np.einsum("kc,khw->chw", wo, dzo)
    skip_grads = {}
    for item in reversed(saved):
        if item[0] == "conv":
            _, name, xin, y = item
            dz = da * (y > 0)
            da, g[name + ".w"], g[name + ".b"] = _conv3x3_backward(xin, P[name + ".w"], dz)
        elif item[0] == "cat":
            _, l, cs = item
            skip_grads[l] = da[:cs]
            d_up = da[cs:]
            da = d_up.reshape(d_up.shape[0], d_up.shape[1] // 2, 2, d_up.shape[2] // 2, 2).sum(axis=(2, 4))
        else:  # pool of level l - 1's output: its window's first maximum, plus the skip path
            _, l, src = item
            da = _maxpool_backward(src, da) + skip_grads.pop(l - 1)
    return loss, g
