"""Pins of the inpainter's definition (oracle/unet.py), tied to arithmetic and closed
forms rather than to the code itself: bfloat16 rounding against an exact-rational
nearest-even rule, the convolution against float64 sums within the FP32 error bound,
pooling and upsampling closed forms, and networks whose weights make the output a
known function of one input channel (which checks the skip order and the wiring)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import unet


def _bf16_exact(v: float) -> float:
    """Nearest bfloat16 by exact rationals: the two neighbours on the 8-bit grid of v's
    binade, the nearer kept, ties to the even last bit."""
    if v == 0 or not np.isfinite(v):
        return v
    m, e = np.frexp(v)  # v = m 2^e, 0.5 <= |m| < 1
    scale = Fr(2) ** (int(e) - 8)  # grid of 8 significant bits
    q = Fr(v) / scale
    lo = q.numerator // q.denominator
    hi = lo + 1
    d_lo, d_hi = q - lo, hi - q
    pick = lo if d_lo < d_hi else hi if d_hi < d_lo else (lo if lo % 2 == 0 else hi)
    return float(pick * scale)


def test_bf16_known_values():
    f = lambda v: float(unet.bf16(np.float32(v)))  # noqa: E731
    assert f(1.0) == 1.0
    assert f(1 + 2**-8) == 1.0                      # a tie goes to the even neighbour
    assert f(1 + 3 * 2**-8) == 1 + 2**-6            # a tie, the even one above
    assert f(1 + 2**-8 + 2**-20) == 1 + 2**-7       # just above the tie
    assert f(-(1 + 3 * 2**-8)) == -(1 + 2**-6)
    assert f(3.0e38) == _bf16_exact(float(np.float32(3.0e38))) < 3.4e38
    assert f(3.4e38) == np.inf                      # past the midpoint above the largest bfloat16
    assert np.isnan(f(np.nan))


def test_bf16_matches_the_exact_rounding_rule():
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(4000) * np.exp2(rng.integers(-30, 30, 4000))).astype(np.float32)
    got = unet.bf16(v)
    for a, g in zip(v, got):
        assert float(g) == _bf16_exact(float(a)), a


def test_conv3x3_within_the_fp32_bound_of_exact_sums():
    rng = np.random.default_rng(1)
    x = unet.bf16(rng.standard_normal((5, 7, 9)).astype(np.float32))
    w = unet.bf16(rng.standard_normal((4, 5, 3, 3)).astype(np.float32))
    b = rng.standard_normal(4).astype(np.float32)
    got = unet.conv3x3(x, w, b)
    xp = np.zeros((5, 9, 11))
    xp[:, 1:-1, 1:-1] = x
    n = 5 * 9 + 1
    for k in range(4):
        for i in range(7):
            for j in range(9):
                terms = [float(w[k, c, dy, dx]) * xp[c, i + dy, j + dx] for c in range(5) for dy in range(3)
                         for dx in range(3)] + [float(b[k])]
                exact = sum(terms)
                bound = n * 2.0**-24 * sum(abs(t) for t in terms)
                assert abs(float(got[k, i, j]) - exact) <= bound


def test_conv1x1_within_the_fp32_bound():
    rng = np.random.default_rng(2)
    x = unet.bf16(rng.standard_normal((6, 4, 4)).astype(np.float32))
    w = unet.bf16(rng.standard_normal((3, 6)).astype(np.float32))
    b = rng.standard_normal(3).astype(np.float32)
    got = unet.conv1x1(x, w, b)
    exact = np.einsum("kc,chw->khw", w.astype(np.float64), x.astype(np.float64)) + b[:, None, None]
    bound = 7 * 2.0**-24 * (np.einsum("kc,chw->khw", np.abs(w.astype(np.float64)), np.abs(x.astype(np.float64)))
                            + np.abs(b)[:, None, None])
    assert (np.abs(got - exact) <= bound).all()


def test_pool_and_upsample_closed_forms():
    x = np.arange(2 * 4 * 6, dtype=np.float32).reshape(2, 4, 6)
    p = unet.maxpool2(x)
    assert p.shape == (2, 2, 3)
    assert p[0, 0, 0] == x[0, 1, 1] and p[1, 1, 2] == x[1, 3, 5]
    u = unet.upsample2(p)
    assert u.shape == (2, 4, 6) and (u[:, ::2, ::2] == p).all() and (u[:, 1::2, 1::2] == p).all()


def test_layer_shapes_follow_the_stated_architecture():
    shapes = dict((n, (w, b)) for n, w, b in unet.layer_shapes())
    assert shapes["enc0a"][0] == (32, 6, 3, 3) and shapes["enc3b"][0] == (256, 256, 3, 3)
    assert shapes["dec2a"][0] == (128, 128 + 256, 3, 3)   # skip (128) then upsampled (256)
    assert shapes["dec0a"][0] == (32, 32 + 64, 3, 3)
    assert shapes["out"][0] == (3, 32)
    assert len(shapes) == 8 + 6 + 1


def _zero_net():
    return {n + s: np.zeros(ws if s == ".w" else bs, np.float32) for n, ws, bs in unet.layer_shapes()
            for s in (".w", ".b")}


def test_zero_network_outputs_one_half():
    p = _zero_net()
    x = np.random.default_rng(3).random((6, 16, 16)).astype(np.float32)
    assert (unet.forward(x, p) == np.float32(0.5)).all()


@pytest.mark.parametrize("path", ["skip", "deep"])
def test_a_channel_routed_through_the_net(path):
    """Weights that carry input channel 0 to the output: through level 0's skip alone, or
    down to level 3 and back up (max pool then nearest upsampling of a 2^3-block-constant
    image returns it).  The output is then sigmoid(2 x0 - 1) with x0 the (BF16) input,
    which pins the order of the concatenation (skip first) and the wiring."""
    p = _zero_net()
    centre = (1, 1)
    p["enc0a.w"][0, 0][centre] = 1.0
    p["enc0b.w"][0, 0][centre] = 1.0
    if path == "deep":
        for l in range(1, 4):
            p[f"enc{l}a.w"][0, 0][centre] = 1.0
            p[f"enc{l}b.w"][0, 0][centre] = 1.0
        for l in (2, 1, 0):
            up = unet.WIDTHS[l]  # the upsampled channels follow the skip's
            p[f"dec{l}a.w"][0, up][centre] = 1.0
            p[f"dec{l}b.w"][0, 0][centre] = 1.0
    else:
        for l in (2, 1, 0):
            p[f"dec{l}a.w"][0, 0][centre] = 1.0 if l == 0 else 0.0
            p[f"dec{l}b.w"][0, 0][centre] = 1.0 if l == 0 else 0.0
    p["out.w"][:, 0] = 2.0
    p["out.b"][:] = -1.0
    rng = np.random.default_rng(4)
    x = np.zeros((6, 16, 24), np.float32)
    blocks = rng.random((2, 3)).astype(np.float32)
    x[0] = np.kron(blocks, np.ones((8, 8), np.float32)) if path == "deep" else rng.random((16, 24))
    x[1:] = rng.random((5, 16, 24))  # other channels carry weight zero
    out = unet.forward(x, p)
    expect = 1.0 / (1.0 + np.exp(-(2.0 * unet.bf16(x[0]).astype(np.float64) - 1.0)))
    assert np.allclose(out, expect[None], rtol=0, atol=2e-7)


def test_compose_keeps_reached_pixels_and_rounds_the_holes():
    warped = np.random.default_rng(5).integers(0, 256, (4, 4, 4), dtype=np.uint8)
    mask = np.zeros((4, 4), np.uint8)
    mask[1, 2] = mask[3, 0] = 1
    color = np.full((3, 4, 4), 0.5, np.float32)
    color[0, 1, 2] = 1.0
    out = unet.compose(warped, mask, color)
    keep = mask == 0
    assert np.array_equal(out[keep], warped[keep])
    assert list(out[1, 2]) == [255, 128, 128, 255]   # 127.5 rounds half to even: 128
    assert list(out[3, 0]) == [128, 128, 128, 255]


def test_input_channels_of_a_tile():
    color = np.full((8, 8, 4), 51, np.uint8)
    color[:, 5:, :3] = 102  # the Patcher's fill at the holes is an input too
    mask = np.zeros((8, 8), np.uint8)
    mask[:, 5:] = 1
    zt = np.full((8, 8), 2.0, np.float32)
    zt[:, 5:] = np.inf
    zsrc = np.full((8, 8), 4.0, np.float32)
    x = unet.tile_input(color, mask, zt, zsrc, near=0.5)
    assert np.allclose(x[0:3, :, :5], 0.2) and np.allclose(x[0:3, :, 5:], 0.4)
    assert (x[3] == mask).all()
    assert np.allclose(x[4, :, :5], 0.25) and (x[4, :, 5:] == 0).all()
    assert np.allclose(x[5], 0.125)


def test_activations_are_rounded_to_bf16_between_layers():
    """Channel 0 through level 0 only, with weights 3, 3, 0.25, 0.25 (all exact in
    bfloat16): each ReLU output is rounded to bfloat16 before the next product, so the
    output is sigmoid(2 a4 - 1) with a1 = r(3 r(x)), a2 = r(3 a1), a3 = r(a2 / 4),
    a4 = r(a3 / 4), r the exact nearest-even rounding to bfloat16."""
    p = _zero_net()
    c = (1, 1)
    p["enc0a.w"][0, 0][c] = 3.0
    p["enc0b.w"][0, 0][c] = 3.0
    p["dec0a.w"][0, 0][c] = 0.25
    p["dec0b.w"][0, 0][c] = 0.25
    p["out.w"][:, 0] = 2.0
    p["out.b"][:] = -1.0
    rng = np.random.default_rng(6)
    x = np.zeros((6, 8, 8), np.float32)
    x[0] = rng.random((8, 8)).astype(np.float32)
    out = unet.forward(x, p)
    r = _bf16_exact
    for i in range(8):
        for j in range(8):
            a1 = r(3.0 * r(float(x[0, i, j])))
            a4 = r(r(r(3.0 * a1) / 4.0) / 4.0)
            expect = 1.0 / (1.0 + np.exp(-(2.0 * a4 - 1.0)))
            assert abs(float(out[0, i, j]) - expect) <= 2e-7
