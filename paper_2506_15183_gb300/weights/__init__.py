"""Parameters of the learned hole inpainter: the layer table, seeded initial weights and
the weights file (a versioned header, then the FP32 parameters).

The network (``include/yoro_unet.h``): encoder levels of 32, 64, 128 and 256 channels with
two 3x3 convolutions each (the first takes the 6 input channels), decoder levels 2, 1, 0
whose first convolution takes the level's skip channels plus the upsampled channels of
the level below, and a 1x1 output layer to 3 colors.  A parameter array holds every layer
in that order, each as its weights (row-major (Cout, Cin, 3, 3), or (3, 32) for the output
layer) followed by its Cout biases.

File ``unet.yw`` (little-endian):  magic ``b"YUNW"``, uint32 version (1), uint32 count of
floats, uint32 CRC-32 of the float bytes, 16 bytes of training metadata (uint32 steps,
uint32 tiles seen in thousands, float32 final training loss, uint32 seed), then the floats.
A reader refuses another magic, version, count or checksum.
"""
from __future__ import annotations

import os
import struct
import zlib

import numpy as np

WIDTHS = (32, 64, 128, 256)
IN_CH = 6
OUT_CH = 3
MAGIC = b"YUNW"
VERSION = 1
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "unet.yw")


def layers():
    """[(name, weight shape, bias count)] in the order of the parameter array."""
    out, cin = [], IN_CH
    for lvl, c in enumerate(WIDTHS):
        out.append((f"enc{lvl}a", (c, cin, 3, 3), c))
        out.append((f"enc{lvl}b", (c, c, 3, 3), c))
        cin = c
    for lvl in (2, 1, 0):
        c = WIDTHS[lvl]
        out.append((f"dec{lvl}a", (c, c + WIDTHS[lvl + 1], 3, 3), c))
        out.append((f"dec{lvl}b", (c, c, 3, 3), c))
    out.append(("out", (OUT_CH, WIDTHS[0]), OUT_CH))
    return out


def count() -> int:
    return sum(int(np.prod(ws)) + nb for _, ws, nb in layers())


def init_params(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, seeded; as one float32 array."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ws, nb in layers():
        fan_in = int(np.prod(ws[1:]))
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), int(np.prod(ws))).astype(np.float32))
        parts.append(np.zeros(nb, np.float32))
    return np.concatenate(parts)


def split(flat: np.ndarray) -> dict:
    """The flat array as {name.w, name.b} arrays (views)."""
    out, o = {}, 0
    for name, ws, nb in layers():
        n = int(np.prod(ws))
        out[name + ".w"] = flat[o:o + n].reshape(ws)
        out[name + ".b"] = flat[o + n:o + n + nb]
        o += n + nb
    return out


def save(flat: np.ndarray, path: str = PATH, steps: int = 0, ktiles: int = 0, loss: float = 0.0,
         seed: int = 0) -> None:
    flat = np.ascontiguousarray(flat, np.float32)
    if flat.size != count():
        raise ValueError(f"expected {count()} parameters, got {flat.size}")
    body = flat.tobytes()
    hdr = MAGIC + struct.pack("<IIIIIfI", VERSION, flat.size, zlib.crc32(body) & 0xFFFFFFFF, steps, ktiles,
                              float(loss), seed)
    tmp = path + ".tmp"
    with open(tmp, "wb") as fh:
        fh.write(hdr + body)
    os.replace(tmp, path)


def read(path: str = PATH):
    """(flat float32 array, metadata dict); raises ValueError on any mismatch."""
    data = open(path, "rb").read()
    if len(data) < 32 or data[:4] != MAGIC:
        raise ValueError("not an inpainter weights file")
    version, n, crc, steps, ktiles, loss, seed = struct.unpack("<IIIIIfI", data[4:32])
    if version != VERSION:
        raise ValueError(f"weights file version {version}, this reader takes {VERSION}")
    if n != count() or len(data) != 32 + 4 * n:
        raise ValueError("weights file has the wrong parameter count")
    body = data[32:]
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError("weights file checksum mismatch")
    return np.frombuffer(body, np.float32).copy(), dict(steps=steps, ktiles=ktiles, loss=loss, seed=seed)


def exists(path: str = PATH) -> bool:
    return os.path.exists(path)


def load_flat(names=None, path: str = PATH) -> np.ndarray:
    flat, _ = read(path)
    if names is not None and list(names) != [n for n, _, _ in layers()]:
        raise ValueError("layer order differs from the weights file's")
    return flat


def flops_per_tile(tile: int = 64) -> int:
    """Multiply-adds x 2 of the network on one tile with the definition's channel counts
    (6 input channels, not the 32 the first layer's memory layout pads them to)."""
    fl = 0
    for name, ws, _ in layers():
        if name == "out":
            fl += 2 * tile * tile * ws[0] * ws[1]
            continue
        side = tile >> int(name[3])
        fl += 2 * side * side * ws[0] * ws[1] * 9
    return fl
