"""Pins of the oracle's general reprojection (Eq. 5 with a general M: a rotated or
vertically offset second eye).

The pins tie oracle.synthesize_pose to things other than itself: the base path (a pure
translation along x with dyadic camera values makes every step exact, so the result is
the base method's byte for byte), the identity pose, a closed form for a vertical
offset over a plane (whole rows move), and, for rotated eyes, the geometry recomputed in
float64: every reached target holds the projection of its source, and no other source
projecting well inside that pixel is nearer.
"""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _dyadic(h, w, seed, run=4):
    rng = np.random.default_rng(seed)
    levels = np.array([0.5, 1.0, 2.0, 4.0, 8.0], np.float32)
    d = np.ascontiguousarray(rng.choice(levels, (h, (w + run - 1) // run)).repeat(run, axis=1)[:, :w])
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    return c, d


@pytest.mark.parametrize("kr,nf", [(3, False), (5, True), (1, False)])
def test_translation_along_x_is_the_base_path(kr, nf):
    for seed in range(3):
        c, d = _dyadic(12, 72, seed)
        fx = fy = 32.0
        for ipd in (0.25, 0.5, 0.0):
            base = oracle.synthesize(c, d, fx, fy, 36.0, 6.0, ipd, 0.05, 1000.0, kernel_rows=kr, nearest_first=nf)
            got = oracle.synthesize_pose(c, d, fx, fy, 36.0, 6.0, np.eye(3), [ipd, 0.0, 0.0], 0.05, 1000.0,
                                         kernel_rows=kr, nearest_first=nf)
            assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])


def test_identity_pose_is_the_identity():
    c, d = _dyadic(9, 40, 7)
    out, mask = oracle.synthesize_pose(c, d, 16.0, 16.0, 20.0, 4.0, np.eye(3), [0.0, 0.0, 0.0], 0.05, 1000.0)
    assert not mask.any() and np.array_equal(out, c)


def test_vertical_offset_over_a_plane_moves_whole_rows():
    """Depth 2, fy = 32, offset 0.25 up: every row moves by fy * 0.25 / 2 = 4 rows; the
    last 4 rows have no source and no reached pixel, so they take the zero fallback."""
    h, w, n = 16, 24, 4
    c, _ = _dyadic(h, w, 3)
    d = np.full((h, w), 2.0, np.float32)
    out, mask = oracle.synthesize_pose(c, d, 32.0, 32.0, 12.0, 8.0, np.eye(3), [0.0, 0.25, 0.0], 0.05, 1000.0)
    assert not mask[: h - n].any() and mask[h - n :].all()
    assert np.array_equal(out[: h - n], c[n:])
    assert not out[h - n :].any()


def _rot(yaw, pitch, roll):
    cy_, sy = np.cos(yaw), np.sin(yaw)
    cp, sp = np.cos(pitch), np.sin(pitch)
    cr, sr = np.cos(roll), np.sin(roll)
    ry = np.array([[cy_, 0, sy], [0, 1, 0], [-sy, 0, cy_]])
    rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    rz = np.array([[cr, -sr, 0], [sr, cr, 0], [0, 0, 1]])
    return (rz @ rx @ ry).astype(np.float32)


@pytest.mark.parametrize("angles,pos", [((0.05, 0.0, 0.0), (0.063, 0.0, 0.0)),
                                        ((0.0, 0.04, 0.02), (0.063, 0.01, 0.0)),
                                        ((-0.03, 0.02, -0.05), (0.05, -0.02, 0.03))])
def test_rotated_eye_matches_the_geometry(angles, pos):
    h, w = 20, 32
    rng = np.random.default_rng(11)
    d = np.repeat(rng.uniform(0.3, 5.0, (h, w // 4)).astype(np.float32), 4, axis=1)
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    fx = fy = 24.0
    cx, cy = w / 2.0, h / 2.0
    rot = _rot(*angles)
    out, mask = oracle.synthesize_pose(c, d, fx, fy, cx, cy, rot, pos, 0.05, 1000.0)
    # float64 projection of every source
    ys, xs = np.mgrid[0:h, 0:w]
    z = d.astype(np.float64)
    p = np.stack([(xs + 0.5 - cx) * z / fx, (ys + 0.5 - cy) * z / fy, z], -1) - np.asarray(pos, np.float64)
    q = p @ rot.astype(np.float64).T
    u = fx * q[..., 0] / q[..., 2] + cx
    v = fy * q[..., 1] / q[..., 2] + cy
    zq = q[..., 2]
    eps = 1e-3
    reached = mask == 0
    assert reached.mean() > 0.5
    # a reached target's color is the color of a source projecting into it (up to
    # rounding), and no source projecting well inside it is nearer than that source
    for ty, tx in zip(*np.nonzero(reached)):
        inside = (u >= tx - eps) & (u < tx + 1 + eps) & (v >= ty - eps) & (v < ty + 1 + eps)
        cand = np.nonzero(inside & (c == out[ty, tx]).all(-1))
        assert cand[0].size > 0, (ty, tx)
        best = zq[cand].min()
        core = (u >= tx + eps) & (u < tx + 1 - eps) & (v >= ty + eps) & (v < ty + 1 - eps)
        if core.any():
            assert best <= zq[core].min() * (1 + 1e-5), (ty, tx)
    # a target that some source projects well inside is reached
    core_hit = np.zeros((h, w), bool)
    iu, iv = np.floor(u).astype(int), np.floor(v).astype(int)
    ok = (u - iu > eps) & (iu + 1 - u > eps) & (v - iv > eps) & (iv + 1 - v > eps) & (zq > 0)
    ok &= (iu >= 0) & (iu < w) & (iv >= 0) & (iv < h)
    core_hit[iv[ok], iu[ok]] = True
    assert reached[core_hit].all()


def test_bad_arguments_are_rejected():
    c, d = _dyadic(2, 8, 1)
    with pytest.raises(RuntimeError):
        oracle.synthesize_pose(c, d, 10.0, 10.0, 4.0, 1.0, np.eye(3), [0.1, 0, 0], 0.05, 1000.0, kernel_rows=2)
