"""Pins of the oracle's row-downsampled intermediate buffer (strategies (c) and (d)).

Each pin ties oracle.synthesize_imb to something other than itself: the base path
(the variant with one cell per pixel and no interpolation is the base method), the
identity at IPD 0, closed forms on a fronto-parallel plane (a whole-pixel shift, and a
half-pixel shift that the linear sampler turns into the rounded mean of two
neighbours), and a plain-Python restatement of the cell warp and the sampling on tiny
rows, compared on the reached pixels (the fill is the base method's, pinned elsewhere).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_15183_gb300 import scene

DIVS = (1, 2, 4, 8, 16)


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()
    scene.build()


def _rand(h, w, seed, zlo=0.3, zhi=6.0, run=5):
    rng = np.random.default_rng(seed)
    runs = rng.uniform(zlo, zhi, (h, (w + run - 1) // run)).astype(np.float32)
    d = np.ascontiguousarray(np.repeat(runs, run, axis=1)[:, :w])
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    return c, d


def test_one_cell_per_pixel_without_interpolation_is_the_base_path():
    cfg = scene.small_config()
    cam = cfg.camera()
    for seed in (1, 2, 3):
        c, d, _ = scene.render(cfg, seed)
        for kr, nf in ((3, False), (5, True), (1, False)):
            ref = oracle.synthesize(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"], cam["near"],
                                    cam["far"], kernel_rows=kr, nearest_first=nf)
            got = oracle.synthesize_imb(c, d, cam["fx"], cam["ipd"], cam["near"], cam["far"], 1, 0,
                                        kernel_rows=kr, nearest_first=nf)
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("div", DIVS)
@pytest.mark.parametrize("interp", (0, 1))
def test_ipd_zero_is_the_identity(div, interp):
    for w in (50, 64, 33):
        c, d = _rand(3, w, w + div)
        out, mask = oracle.synthesize_imb(c, d, 40.0, 0.0, 0.05, 1000.0, div, interp)
        assert not mask.any()
        assert np.array_equal(out, c)


@pytest.mark.parametrize("div", DIVS)
@pytest.mark.parametrize("interp", (0, 1))
def test_plane_with_a_whole_pixel_shift(div, interp):
    """Depth 2 and k = fx ipd = 32: every cell shifts by exactly 16 pixels.  Pixel x shows
    source x + 16; the last 16 pixels of a row are holes, filled by the fallback with
    the last reached pixel's color, source w - 1."""
    h, w, n = 3, 96, 16
    c, _ = _rand(h, w, 5)
    d = np.full((h, w), 2.0, np.float32)
    out, mask = oracle.synthesize_imb(c, d, 64.0, 0.5, 0.05, 1000.0, div, interp)
    assert not mask[:, : w - n].any() and mask[:, w - n :].all()
    assert np.array_equal(out[:, : w - n], c[:, n:])
    assert np.array_equal(out[:, w - n :], np.repeat(c[:, w - 1 : w], n, axis=1))


@pytest.mark.parametrize("div", DIVS)
def test_plane_with_a_half_pixel_shift_blends_two_neighbours(div):
    """k = 33, depth 2: a shift of 16.5.  Without interpolation a pixel copies its place
    in the winning cell; with it the linear sampler lands halfway between sources
    x + 16 and x + 17: (c0 + c1) / 2, rounded half to even."""
    h, w = 2, 96
    c, _ = _rand(h, w, 9)
    d = np.full((h, w), 2.0, np.float32)
    out, mask = oracle.synthesize_imb(c, d, 66.0, 0.5, 0.05, 1000.0, div, 1)
    ok = ~mask.astype(bool)
    c0 = c[:, 16:-1].astype(np.int32)
    c1 = c[:, 17:].astype(np.int32)
    mean = np.rint((c0 + c1) / 2.0).astype(np.uint8)  # numpy rounds half to even
    x = np.arange(w - 17)
    sel = ok[:, x]
    assert sel.sum() > 0
    assert np.array_equal(out[:, x][sel], mean[sel])


def _py_warped(c, d, fx, ipd, near, far, div, interp):
    """Steps 1-3 of the reading restated in plain Python with binary32 rounding."""
    f32 = np.float32
    h, w = d.shape
    ws = (w + div - 1) // div
    k = f32(f32(fx) * f32(ipd))
    mask = np.ones((h, w), np.uint8)
    out = np.zeros((h, w, 4), np.uint8)
    for y in range(h):
        win, wz, wd = [-1] * ws, [None] * ws, [None] * ws
        for i in range(ws):
            p = min(div * i + div // 2, w - 1)
            z = f32(d[y, p])
            if not z > 0 or math.isinf(z):
                z = f32(far)
            zc = f32(min(max(z, f32(near)), f32(far)))
            disp = f32(k / zc)
            t = f32(f32(f32(p) + f32(0.5)) - disp)
            tc = math.floor(t / div)
            if 0 <= tc < ws and (win[tc] < 0 or zc < wz[tc]):
                win[tc], wz[tc], wd[tc] = i, zc, disp
        for x in range(w):
            j = x // div
            if win[j] < 0:
                continue
            mask[y, x] = 0
            if not interp:
                out[y, x] = c[y, min(div * win[j] + x - div * j, w - 1)]
                continue
            off = (x + 0.5) - (div * j + div / 2)
            nb = j - 1 if off < 0 else j + 1
            D = wd[j]
            if off != 0 and 0 <= nb < ws and win[nb] >= 0:
                D = f32(wd[j] + f32(f32(wd[nb] - wd[j]) * f32(abs(off) / div)))
            u = f32(f32(x) + D)
            if u <= 0:
                out[y, x] = c[y, 0]
            elif u >= w - 1:
                out[y, x] = c[y, w - 1]
            else:
                i0 = math.floor(u)
                fr = f32(u - f32(i0))
                for ch in range(4):
                    c0, c1 = f32(c[y, i0, ch]), f32(c[y, i0 + 1, ch])
                    out[y, x, ch] = int(np.rint(f32(c0 + f32(f32(c1 - c0) * fr))))
    return out, mask


@pytest.mark.parametrize("div", DIVS)
@pytest.mark.parametrize("interp", (0, 1))
def test_restated_cell_warp_and_sampling_on_tiny_rows(div, interp):
    for seed in range(4):
        w = 20 + 7 * seed
        c, d = _rand(2, w, 100 * div + seed, zlo=0.2, zhi=3.0, run=3)
        fx, ipd = 12.0, 0.4
        ref_out, ref_mask = _py_warped(c, d, fx, ipd, 0.05, 1000.0, div, interp)
        out, mask = oracle.synthesize_imb(c, d, fx, ipd, 0.05, 1000.0, div, interp)
        assert np.array_equal(mask, ref_mask)
        reached = mask == 0
        assert np.array_equal(out[reached], ref_out[reached])


def test_bad_arguments_are_rejected():
    c, d = _rand(2, 8, 1)
    for div, interp in ((3, 0), (0, 0), (32, 0), (-2, 1)):
        with pytest.raises(RuntimeError):
            oracle.synthesize_imb(c, d, 10.0, 0.1, 0.05, 1000.0, div, interp)
