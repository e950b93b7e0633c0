"""Image-quality measures of a synthesized eye against the analytic ground truth, over the
hole pixels (the disocclusions a fill invents).

* ``psnr``: 10 log10(255^2 / MSE), the MSE over the masked pixels' R, G and B values.
* ``ssim_gaussian``: the structural similarity of Wang et al. with an 11 x 11 Gaussian
  window (sigma 1.5), constants C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = 255, computed per
  color channel with symmetric (mirror) padding at the image border; the SSIM map of each
  channel is averaged over the masked pixels, then over the channels.
* ``ssim_global``: the form the paper's evaluation prints (Sec. Evaluation): the same
  expression with the means, variances and covariance taken over all masked pixels at
  once, averaged over the channels.

The paper's own averages (34.09 dB, 0.9679) are over whole images of its scenes against
rendered ground truth; these functions report the hole pixels only.
"""
from __future__ import annotations

import numpy as np

L = 255.0
C1 = (0.01 * L) ** 2
C2 = (0.03 * L) ** 2


def _rgb(a):
    a = np.asarray(a)
    return a[..., :3].astype(np.float64)


def psnr(a, b, mask=None) -> float:
    x, y = _rgb(a), _rgb(b)
    m = np.ones(x.shape[:2], bool) if mask is None else np.asarray(mask).astype(bool)
    if not m.any():
        return float("nan")
    mse = float(((x[m] - y[m]) ** 2).mean())
    return float("inf") if mse == 0.0 else 10.0 * np.log10(L * L / mse)


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    r = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    return g / g.sum()


def _filter(img, g):
    """Separable correlation with g along both axes, mirror padding."""
    r = len(g) // 2
    p = np.pad(img, r, mode="symmetric")
    tmp = sum(g[k] * p[k:k + img.shape[0], :] for k in range(len(g)))
    return sum(g[k] * tmp[:, k:k + img.shape[1]] for k in range(len(g)))


def ssim_map(x, y, size: int = 11, sigma: float = 1.5) -> np.ndarray:
    """SSIM map of two single-channel float images."""
    g = gaussian_window(size, sigma)
    mx, my = _filter(x, g), _filter(y, g)
    sxx = _filter(x * x, g) - mx * mx
    syy = _filter(y * y, g) - my * my
    sxy = _filter(x * y, g) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim_gaussian(a, b, mask=None) -> float:
    x, y = _rgb(a), _rgb(b)
    m = np.ones(x.shape[:2], bool) if mask is None else np.asarray(mask).astype(bool)
    if not m.any():
        return float("nan")
    return float(np.mean([ssim_map(x[..., c], y[..., c])[m].mean() for c in range(3)]))


def ssim_global(a, b, mask=None) -> float:
    x, y = _rgb(a), _rgb(b)
    m = np.ones(x.shape[:2], bool) if mask is None else np.asarray(mask).astype(bool)
    if not m.any():
        return float("nan")
    vals = []
    for c in range(3):
        u, v = x[..., c][m], y[..., c][m]
        mu, mv = u.mean(), v.mean()
        su, sv, suv = u.var(), v.var(), ((u - mu) * (v - mv)).mean()
        vals.append(((2 * mu * mv + C1) * (2 * suv + C2)) / ((mu * mu + mv * mv + C1) * (su + sv + C2)))
    return float(np.mean(vals))
