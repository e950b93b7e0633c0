"""Hole-quality measures (paper_2506_15183_gb300/quality.py), pinned by closed forms and
a brute-force window sum."""
import numpy as np

from paper_2506_15183_gb300 import quality as Q


def _img(seed, h=24, w=20):
    return np.random.default_rng(seed).integers(0, 256, (h, w, 4)).astype(np.uint8)


def test_psnr_closed_forms():
    a = _img(1)
    assert Q.psnr(a, a) == float("inf")
    b = a.astype(int)
    b[..., :3] = np.clip(b[..., :3], 0, 250) + 5  # every color value off by exactly 5
    assert abs(Q.psnr(a.clip(0, 250), b.astype(np.uint8)) - 20 * np.log10(255 / 5)) < 1e-12
    # only masked pixels count; alpha never does
    m = np.zeros(a.shape[:2], bool)
    m[3:7, 2:9] = True
    c = a.copy()
    c[~m] = 0
    c[..., 3] = 17
    assert Q.psnr(a, c, m) == float("inf")


def test_ssim_of_an_image_with_itself_is_one():
    a = _img(2)
    assert abs(Q.ssim_gaussian(a, a) - 1.0) < 1e-12
    assert abs(Q.ssim_global(a, a) - 1.0) < 1e-12


def test_ssim_global_closed_forms():
    """A constant shift c keeps the structure term at 1: SSIM = (2 mu (mu + c) + C1) /
    (mu^2 + (mu + c)^2 + C1).  Inverting about the mean keeps the luminance term at 1:
    SSIM = (C2 - 2 var) / (2 var + C2)."""
    rng = np.random.default_rng(3)
    x = rng.integers(20, 200, (16, 16)).astype(np.float64)
    a = np.repeat(x[..., None], 3, axis=2)
    mu, var = x.mean(), x.var()
    c = 30.0
    want = (2 * mu * (mu + c) + Q.C1) / (mu * mu + (mu + c) ** 2 + Q.C1)
    assert abs(Q.ssim_global(a, a + c) - want) < 1e-12
    inv = 2 * mu - a
    assert abs(Q.ssim_global(a, inv) - (Q.C2 - 2 * var) / (2 * var + Q.C2)) < 1e-12


def test_gaussian_ssim_map_equals_a_brute_force_window_sum():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 255, (15, 13))
    y = np.clip(x + rng.normal(0, 20, x.shape), 0, 255)
    g = Q.gaussian_window()
    g2 = np.outer(g, g)
    xp, yp = np.pad(x, 5, mode="symmetric"), np.pad(y, 5, mode="symmetric")
    want = np.empty_like(x)
    for i in range(x.shape[0]):
        for j in range(x.shape[1]):
            wx, wy = xp[i:i + 11, j:j + 11], yp[i:i + 11, j:j + 11]
            mx, my = (g2 * wx).sum(), (g2 * wy).sum()
            sxx = (g2 * wx * wx).sum() - mx * mx
            syy = (g2 * wy * wy).sum() - my * my
            sxy = (g2 * wx * wy).sum() - mx * my
            want[i, j] = ((2 * mx * my + Q.C1) * (2 * sxy + Q.C2)) / ((mx * mx + my * my + Q.C1) * (sxx + syy + Q.C2))
    assert np.allclose(Q.ssim_map(x, y), want, rtol=0, atol=1e-12)
    assert abs(g.sum() - 1) < 1e-15 and abs(g[5] / g[4] - np.exp(1 / (2 * 1.5 ** 2))) < 1e-12


def test_ssim_is_symmetric_and_at_most_one():
    a, b = _img(5), _img(6)
    assert abs(Q.ssim_gaussian(a, b) - Q.ssim_gaussian(b, a)) < 1e-12
    assert Q.ssim_gaussian(a, b) < 1 and Q.ssim_global(a, b) < 1
