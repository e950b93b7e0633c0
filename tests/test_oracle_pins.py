"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms of
the method (IPD = 0, a fronto-parallel plane, the geometric form of Eq. 6's
recursion), brute force on tiny inputs (nearest-wins, hole edges), an analytic
ray-cast of the true second eye, and a worked example computed by hand.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2506_15183_gb300 import scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- disparity
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ipd_zero_is_identity(seed):
    """IPD = 0: disp = 0 and floor(x + 0.5) = x, so the right eye equals the left eye."""
    cfg = scene.small_config()
    c, d, _ = scene.render(cfg, seed)
    out, mask = oracle.synthesize(c, d, cfg.fx, cfg.fy, cfg.cx, cfg.cy, 0.0, cfg.near, cfg.far)
    assert np.array_equal(out, c)
    assert not mask.any()


def test_ipd_zero_identity_with_invalid_depths():
    rng = np.random.default_rng(7)
    h, w = 5, 37
    d = rng.uniform(0.01, 50, (h, w)).astype(np.float32)
    d.flat[::5] = 0.0
    d.flat[1::7] = -3.0
    d.flat[2::11] = np.nan
    d.flat[3::13] = np.inf
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    out, mask = oracle.synthesize(c, d, 20.0, 20.0, 18.5, 2.5, 0.0, 0.05, 1000.0)
    assert np.array_equal(out, c) and not mask.any()


def _plane(h, w, z):
    rng = np.random.default_rng(h * 1000 + w)
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    return c, np.full((h, w), z, np.float32)


@pytest.mark.parametrize("s,frac,expect_shift", [(3, 0.25, 3), (3, 0.75, 4), (0, 0.25, 0), (7, 0.4, 7)])
def test_fronto_parallel_plane_constant_shift(s, frac, expect_shift):
    """A plane at depth Z moves every pixel by the same amount: x_R = floor(x + 0.5 - k/Z).

    With k/Z = s + frac, the shift is s for frac < 0.5 and s + 1 for frac > 0.5.  Targets
    no source reaches are the last `shift` columns; they have no background edge
    (R = W), so the fallback copies their left neighbour, i.e. the last source column.
    fx != fy checks that the horizontal focal length is the one used.
    """
    h, w = 6, 48
    fx, fy, ipd = 40.0, 55.0, 0.1
    k = np.float32(fx) * np.float32(ipd)
    z = float(np.float32(k / np.float32(s + frac)))
    c, d = _plane(h, w, z)
    out, mask = oracle.synthesize(c, d, fx, fy, w / 2, h / 2, ipd, 0.05, 1000.0)
    cols = np.minimum(np.arange(w) + expect_shift, w - 1)
    assert np.array_equal(out, c[:, cols])
    assert np.array_equal(mask, np.broadcast_to(np.arange(w) >= w - expect_shift, (h, w)).astype(np.uint8))


def test_near_and_far_clamp():
    """Depths below near behave as near; zero, negative, NaN and inf behave as far."""
    h, w = 3, 40
    fx, ipd, near, far = 40.0, 0.1, 0.5, 40.0
    c, _ = _plane(h, w, 1.0)
    d_near = np.full((h, w), 0.01, np.float32)
    ref, _ = oracle.synthesize(c, np.full((h, w), near, np.float32), fx, fx, 20, 1.5, ipd, near, far)
    out, _ = oracle.synthesize(c, d_near, fx, fx, 20, 1.5, ipd, near, far)
    assert np.array_equal(out, ref)
    ref_far, _ = oracle.synthesize(c, np.full((h, w), far, np.float32), fx, fx, 20, 1.5, ipd, near, far)
    for bad in (0.0, -2.0, np.nan, np.inf, 5000.0):
        out, _ = oracle.synthesize(c, np.full((h, w), bad, np.float32), fx, fx, 20, 1.5, ipd, near, far)
        assert np.array_equal(out, ref_far), bad
    xt, zc = oracle.disparity(np.array([[0.01, np.nan, 7.0, 90.0]], np.float32), fx, ipd, near, far)
    assert zc.tolist() == [[near, far, 7.0, far]]


def test_off_frame_targets_are_dropped():
    """A source whose shifted centre lands left of column 0 (t in (-1, 0)) is dropped."""
    fx, ipd = 40.0, 0.1  # k = 4
    d = np.full((1, 8), np.float32(4.0 / 3.25), np.float32)  # disp = 3.25
    xt, _ = oracle.disparity(d, fx, ipd, 0.05, 1000.0)
    assert xt.tolist() == [[-1, -1, -1, 0, 1, 2, 3, 4]]


# ----------------------------------------------------------------------------- forward warp
@pytest.mark.parametrize("seed", range(6))
def test_nearer_wins_brute_force(seed):
    """Every reached target holds argmin over the sources mapped there of (depth, column)."""
    rng = np.random.default_rng(seed)
    h, w = 4, 16
    fx, ipd = 8.0, 0.5  # k = 4: disparities of several pixels at depth ~1
    d = rng.choice(np.array([0.6, 0.8, 1.0, 1.3, 2.0, 4.0, 9.0], np.float32), (h, w))
    xt, zc = oracle.disparity(d, fx, ipd, 0.05, 1000.0)
    src, zt = oracle.forward_warp(xt, zc)
    for y in range(h):
        for t in range(w):
            cands = [x for x in range(w) if xt[y, x] == t]
            if not cands:
                assert src[y, t] == -1 and np.isinf(zt[y, t])
                continue
            best = min(cands, key=lambda x: (float(zc[y, x]), x))
            assert src[y, t] == best
            assert zt[y, t] == zc[y, best]


def test_equal_depth_tie_goes_to_lowest_source_column():
    xt = np.array([[2, 2, 2, 0, -1]], np.int32)
    zc = np.array([[5.0, 5.0, 3.0, 1.0, 1.0]], np.float32)
    src, zt = oracle.forward_warp(xt, zc)
    assert src.tolist() == [[3, -1, 2, -1, -1]]
    xt = np.array([[1, 1, 1]], np.int32)
    zc = np.array([[2.0, 2.0, 2.0]], np.float32)
    src, _ = oracle.forward_warp(xt, zc)
    assert src.tolist() == [[-1, 0, -1]]


def _rightmost_sources(xt):
    """For every target of every row, the largest source column mapped there (-1: none)."""
    h, w = xt.shape
    right = np.full(h * w, -1, np.int64)
    ys, xs = np.nonzero((xt >= 0) & (xt < w))
    np.maximum.at(right, ys * w + xt[ys, xs], xs)
    return right.reshape(h, w)


def _hostile_depths(rng, h, w, zlo, zhi):
    d = np.empty((h, w), np.float32)
    for y in range(h):
        x = 0
        while x < w:
            run = int(rng.integers(1, 30))
            d[y, x : x + run] = rng.uniform(zlo, zhi)
            x += run
    d *= rng.uniform(0.97, 1.03, (h, w)).astype(np.float32)
    flat = d.reshape(-1)
    idx = rng.choice(flat.size, size=flat.size // 20, replace=False)
    special = np.array([0.0, -0.0, -1.0, np.nan, np.inf, -np.inf, 1e-40, 1e-3, 1e7], np.float32)
    flat[idx] = rng.choice(special, idx.size)
    return d


@pytest.mark.parametrize("case", range(8))
def test_nearest_source_is_the_rightmost_one(case):
    """Two sources of a row that reach the same target: the one further right is nearer.

    With k = fx * ipd >= 0, Q = RN(k / zc) does not grow with zc, and floor(RN(x + 0.5 - Q))
    rises by at least one per column for targets >= 0, so sources of equal clamped depth
    never meet on a target and, where two meet, the right one has the larger Q, i.e. the
    smaller depth.  The nearest-wins z-test of Alg. 2 therefore keeps the rightmost
    source and its tie rule never decides.  Checked by brute force on the method's own
    target columns: wide disparities, both clamps, invalid depths, repeated depths, and
    depths whose disparity sits next to a rounding boundary of the target column.
    """
    rng = np.random.default_rng(900 + case)
    h, w = 12, 301
    fx, ipd, near, far = [(150.0, 0.063, 0.05, 1000.0), (8.0, 0.5, 0.05, 1000.0), (150.0, 0.3, 0.2, 5.0),
                          (916.0, 0.063, 0.05, 1000.0)][case % 4]
    if case < 4:
        d = _hostile_depths(rng, h, w, 0.01, 60.0)
    else:  # disparities k/z = n + 1/2 + tiny: targets next to a floor boundary
        k = np.float32(fx) * np.float32(ipd)
        n = rng.integers(0, 60, (h, w)).astype(np.float64)
        eps = rng.choice(np.array([-1e-6, -1e-7, 0.0, 1e-7, 1e-6]), (h, w))
        d = (float(k) / (n + 0.5 + eps)).astype(np.float32)
        d[:, ::17] = d[:, 1::17][:, : d[:, ::17].shape[1]]  # repeated depths side by side
    xt, zc = oracle.disparity(d, fx, ipd, near, far)
    src, _ = oracle.forward_warp(xt, zc)
    assert np.array_equal(src, _rightmost_sources(xt))
    for y in range(h):  # equal clamped depth never shares a target
        ok = (xt[y] >= 0) & (xt[y] < w)
        pairs = set(zip(xt[y][ok].tolist(), zc[y][ok].view(np.uint32).tolist()))
        assert len(pairs) == int(ok.sum())


def test_nearest_source_is_the_rightmost_one_on_the_workload():
    """The same property on a 1832x1920 frame of the scene generator (200 primitives)."""
    cfg = scene.quest_config()
    _, d, _ = scene.render(cfg, 2)
    xt, zc = oracle.disparity(d, cfg.fx, cfg.ipd, cfg.near, cfg.far)
    src, _ = oracle.forward_warp(xt, zc)
    assert np.array_equal(src, _rightmost_sources(xt))


# ----------------------------------------------------------------------------- hole edges
@pytest.mark.parametrize("seed", range(4))
def test_hole_edges_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    h, w = 5, 23
    src = np.where(rng.random((h, w)) < 0.45, 0, -1).astype(np.int32)
    src[0] = -1  # a row with no reached pixel
    L, R = oracle.hole_edges(src)
    for y in range(h):
        for u in range(w):
            if src[y, u] >= 0:
                continue
            left = [x for x in range(u) if src[y, x] >= 0]
            right = [x for x in range(u + 1, w) if src[y, x] >= 0]
            assert L[y, u] == (max(left) if left else -1)
            assert R[y, u] == (min(right) if right else w)


# ----------------------------------------------------------------------------- fill
def _fill_case(valid, zt, colors, kernel_rows=3, nearest_first=False):
    src = np.where(valid, 0, -1).astype(np.int32)
    L, R = oracle.hole_edges(src)
    warped = np.where(valid[..., None], colors, 0).astype(np.uint8)
    return oracle.fill(src, zt.astype(np.float32), L, R, warped, kernel_rows, nearest_first), L, R


def test_fill_golden_two_contributors():
    """Worked example of Algorithm 3 / Eq. 6 with two contributors (computed by hand)."""
    g = json.load(open(os.path.join(GOLDEN, "fill_two_contributors.json")))
    w = 12
    valid = np.array([[1, 1, 1, 0, 0, 1, 0, 0, 1, 1, 1, 1]], bool)
    zt = np.where(valid, 10.0, np.inf)
    zt[0, :3] = 1.0  # occluder on the left edge
    colors = np.zeros((1, w, 4), np.uint8)
    colors[0, 8] = g["c1"]  # column R + w = 5 + 3: visited first
    colors[0, 5] = g["c2"]  # column R: visited last
    colors[0, 9:] = 33      # beyond R + w: outside the kernel
    colors[0, :3] = 250     # occluder side: never sampled
    out, L, R = _fill_case(valid, zt, colors)
    assert L[0, 3] == 2 and R[0, 3] == 5
    by_t = {Fraction(cs["t_num"], cs["t_den"]): cs for cs in g["cases"]}
    # u = 3: t = (5 - 3) / 3 = 2/3; u = 4: t = 1/3
    assert out[0, 3].tolist() == by_t[Fraction(2, 3)]["expected"]
    assert out[0, 4].tolist() == by_t[Fraction(1, 3)]["expected"]


def _expected_fill(valid, zt, colors, v, u, kernel_rows=3, nearest_first=False):
    """Closed form of Algorithm 3 + Eq. 6 (exact rationals) for hole pixel (v, u).

    With q = 1/2 - 3t/10, the i-th contributor (0-based, in kernel order) receives
    weight q^i (1 - q), so the result is sum q^i c_i / sum q^i.  Returns (value list
    of Fractions, or None for the fallback, list of fallback bytes).
    """
    h, w = valid.shape
    left = [x for x in range(u) if valid[v, x]]
    right = [x for x in range(u + 1, w) if valid[v, x]]
    L = max(left) if left else -1
    R = min(right) if right else w
    if R < w:
        fb = colors[v, R]
    elif L >= 0:
        fb = colors[v, L]
    else:
        fb = np.zeros(4, np.uint8)
    if R == w:
        return None, fb
    wd = R - L
    d_occ = zt[v, L] if L >= 0 else 0.0
    t = Fraction(R - u, wd)
    q = Fraction(1, 2) - Fraction(3, 10) * t
    contrib = []
    hr = (kernel_rows - 1) // 2
    for vv in range(v - hr, v + hr + 1):
        if not 0 <= vv < h:
            continue
        cols = range(min(R + wd, w - 1), R - 1, -1)
        for j in (reversed(cols) if nearest_first else cols):
            if valid[vv, j] and not zt[vv, j] < d_occ:
                contrib.append(colors[vv, j])
    if not contrib:
        return None, fb
    num = [Fraction(0)] * 4
    den = Fraction(0)
    for i, col in enumerate(contrib):
        wi = q ** i
        den += wi
        for ch in range(4):
            num[ch] += wi * int(col[ch])
    return [n / den for n in num], fb


@pytest.mark.parametrize("seed", range(8))
def test_fill_matches_geometric_closed_form(seed):
    """Random small scenes: every hole pixel equals the closed form (or its fallback)."""
    rng = np.random.default_rng(1000 + seed)
    h, w = 4, 30
    valid = rng.random((h, w)) < 0.6
    zt = rng.choice(np.array([1.0, 2.0, 5.0, 5.0, 9.0]), (h, w)).astype(np.float32)
    zt = np.where(valid, zt, np.inf).astype(np.float32)
    colors = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    out, _, _ = _fill_case(valid, zt, colors)
    checked = 0
    for v in range(h):
        for u in range(w):
            if valid[v, u]:
                assert out[v, u].tolist() == colors[v, u].tolist()
                continue
            exact, fb = _expected_fill(valid, zt, colors, v, u)
            if exact is None:
                assert out[v, u].tolist() == fb.tolist()
                continue
            for ch in range(4):
                e = exact[ch]
                frac = e - int(e)
                if abs(frac - Fraction(1, 2)) < Fraction(1, 100):
                    continue  # too close to a rounding tie for binary32 to decide like exact math
                assert out[v, u, ch] == int(e + Fraction(1, 2)), (v, u, ch, float(e))
                checked += 1
    assert checked > 50


@pytest.mark.parametrize("kernel_rows,nearest_first", [(1, False), (1, True), (3, True), (5, False), (5, True),
                                                      (7, False)])
def test_fill_variants_match_geometric_closed_form(kernel_rows, nearest_first):
    """The Patcher's variants (kernel height h, nearest-first column order): every hole
    pixel equals the closed form sum q^i c_i / sum q^i over its kernel (or the fallback)."""
    rng = np.random.default_rng(2000 + kernel_rows * 2 + int(nearest_first))
    h, w = 9, 30
    valid = rng.random((h, w)) < 0.6
    zt = rng.choice(np.array([1.0, 2.0, 5.0, 5.0, 9.0]), (h, w)).astype(np.float32)
    zt = np.where(valid, zt, np.inf).astype(np.float32)
    colors = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    out, _, _ = _fill_case(valid, zt, colors, kernel_rows, nearest_first)
    checked = 0
    for v in range(h):
        for u in range(w):
            if valid[v, u]:
                continue
            exact, fb = _expected_fill(valid, zt, colors, v, u, kernel_rows, nearest_first)
            if exact is None:
                assert out[v, u].tolist() == fb.tolist()
                continue
            for ch in range(4):
                e = exact[ch]
                if abs(e - int(e) - Fraction(1, 2)) < Fraction(1, 100):
                    continue  # too close to a rounding tie for binary32 to decide like exact math
                assert out[v, u, ch] == int(e + Fraction(1, 2)), (v, u, ch, float(e))
                checked += 1
    assert checked > 100


def test_fill_kernel_height_selects_the_rows():
    """h = 1 reads row v only; h = 5 reaches rows v - 2 and v + 2, which h = 3 does not."""
    h, w = 7, 20
    v, L, R = 3, 4, 7  # hole at 5, 6 of row 3; kernel columns 10..7
    valid = np.zeros((h, w), bool)
    valid[:, : L + 1] = True
    valid[v, R] = True           # the only contributor of row v
    valid[v - 1, 8] = True       # rows v -+ 1: reached by h >= 3
    valid[v + 2, 9] = True       # row v + 2: reached by h >= 5 only
    zt = np.where(valid, 4.0, np.inf).astype(np.float32)
    colors = np.zeros((h, w, 4), np.uint8)
    colors[v, R] = (10, 20, 30, 255)
    colors[v - 1, 8] = (200, 0, 0, 255)
    colors[v + 2, 9] = (0, 0, 250, 255)
    out1, _, _ = _fill_case(valid, zt, colors, kernel_rows=1)
    assert out1[v, 5].tolist() == [10, 20, 30, 255]  # one contributor returns its color
    out3, _, _ = _fill_case(valid, zt, colors, kernel_rows=3)
    out5, _, _ = _fill_case(valid, zt, colors, kernel_rows=5)
    assert out3[v, 5].tolist() != out1[v, 5].tolist()
    assert out5[v, 5].tolist() != out3[v, 5].tolist()
    # rows v-1..v+1 hold no contributor (R itself is nearer than the occluder): h = 3 falls
    # back to the color at (v, R), h = 5 returns row v+2's color alone
    valid2 = np.zeros((h, w), bool)
    valid2[:, : L + 1] = True
    valid2[v, R] = True
    valid2[v + 2, 9] = True
    zt2 = np.full((h, w), 5.0, np.float32)
    zt2[v, R] = 1.0   # foreground: skipped by the depth gate
    zt2[v + 2, 9] = 8.0
    zt2 = np.where(valid2, zt2, np.inf).astype(np.float32)
    colors2 = np.zeros((h, w, 4), np.uint8)
    colors2[v, R] = (9, 9, 9, 255)
    colors2[v + 2, 9] = (0, 0, 250, 255)
    out_a, _, _ = _fill_case(valid2, zt2, colors2, kernel_rows=3)
    out_b, _, _ = _fill_case(valid2, zt2, colors2, kernel_rows=5)
    assert out_a[v, 5].tolist() == [9, 9, 9, 255]
    assert out_b[v, 5].tolist() == [0, 0, 250, 255]


def test_fill_column_order_changes_the_first_weight():
    """Two contributors a (at R) and b (at R + 1) in a one-row kernel: the first one visited
    gets weight 1 - q, the second q (1 - q), so the result is (c0 + q c1) / (1 + q) with c0
    the first: b for the paper's farthest-first order, a for nearest-first."""
    w = 12
    L, R = 2, 5  # holes at 3, 4; w = 3, kernel columns 8..5
    valid = np.zeros((1, w), bool)
    valid[0, : L + 1] = True
    valid[0, R] = valid[0, R + 1] = True
    zt = np.where(valid, 4.0, np.inf).astype(np.float32)
    colors = np.zeros((1, w, 4), np.uint8)
    a, b = np.array([200, 10, 90, 255]), np.array([20, 230, 60, 255])
    colors[0, R], colors[0, R + 1] = a, b
    for nearest_first, first, second in ((False, b, a), (True, a, b)):
        out, _, _ = _fill_case(valid, zt, colors, kernel_rows=1, nearest_first=nearest_first)
        for u in (3, 4):
            t = Fraction(R - u, R - L)
            q = Fraction(1, 2) - Fraction(3, 10) * t
            for ch in range(4):
                e = (int(first[ch]) + q * int(second[ch])) / (1 + q)
                assert out[0, u, ch] == int(e + Fraction(1, 2)), (nearest_first, u, ch)


@pytest.mark.parametrize("t_num,t_den", [(1, 2), (1, 7), (6, 7), (4, 5)])
def test_fill_single_contributor_returns_its_color(t_num, t_den):
    """One contributor: acc = c w and den = w, so the result is c exactly."""
    rng = np.random.default_rng(t_num * 10 + t_den)
    w = 30
    for _ in range(20):
        col = rng.integers(0, 256, 4)
        # hole of width t_den - 1 ending at R; only R contributes (the rest of the kernel are holes)
        L = 3
        R = L + t_den
        valid = np.zeros((1, w), bool)
        valid[0, : L + 1] = True
        valid[0, R] = True
        zt = np.where(valid, 4.0, np.inf)
        colors = np.zeros((1, w, 4), np.uint8)
        colors[0, R] = col
        out, _, _ = _fill_case(valid, zt, colors)
        u = R - t_num
        assert out[0, u].tolist() == col.tolist()


def test_fill_constant_color_long_run():
    """Two hundred contributors of one color give that color (weights normalised by 1 - wrem)."""
    h, w = 3, 420
    valid = np.ones((h, w), bool)
    valid[1, 10:210] = False  # hole of width 201 in the middle row: L = 9, R = 210
    zt = np.where(valid, 3.0, np.inf)
    colors = np.zeros((h, w, 4), np.uint8)
    colors[:] = (17, 200, 91, 255)
    out, _, _ = _fill_case(valid, zt, colors)
    assert (out[1, 10:210] == np.array([17, 200, 91, 255], np.uint8)).all()


def test_fill_depth_gate_and_extent():
    """Foreground candidates (nearer than the occluder) and pixels outside the kernel do not count."""
    h, w = 5, 24
    valid = np.ones((h, w), bool)
    v, L, R = 2, 5, 8  # holes at 6, 7 of row 2; w = 3; kernel columns 11..8, rows 1..3
    valid[v, L + 1 : R] = False
    zt = np.full((h, w), 6.0, np.float32)
    zt[v, L] = 2.0  # occluder depth
    zt = np.where(valid, zt, np.inf).astype(np.float32)
    rng = np.random.default_rng(3)
    colors = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    base, _, _ = _fill_case(valid, zt, colors)

    def changed(mod):
        c2 = colors.copy()
        z2 = zt.copy()
        mod(c2, z2)
        o, _, _ = _fill_case(valid, z2, c2)
        return not np.array_equal(o[v, L + 1 : R], base[v, L + 1 : R])

    # outside the kernel: rows v +- 2, column R + w + 1, the occluder side
    assert not changed(lambda c, z: c.__setitem__((0, 9), 255 - c[0, 9]))
    assert not changed(lambda c, z: c.__setitem__((4, 9), 255 - c[4, 9]))
    assert not changed(lambda c, z: c.__setitem__((v, 12), 255 - c[v, 12]))
    assert not changed(lambda c, z: c.__setitem__((v, 4), 255 - c[v, 4]))
    # inside the kernel, farthest corner and nearest column
    assert changed(lambda c, z: c.__setitem__((1, 11), 255 - c[1, 11]))
    assert changed(lambda c, z: c.__setitem__((1, 8), 255 - c[1, 8]))

    # a foreground candidate strictly nearer than the occluder is skipped...
    def fg(c, z):
        z[1, 11] = 1.5
        c[1, 11] = 255 - c[1, 11]

    def fg_ref(c, z):
        z[1, 11] = 1.5

    c_a, z_a = colors.copy(), zt.copy()
    fg_ref(c_a, z_a)
    ref, _, _ = _fill_case(valid, z_a, c_a)
    c_b, z_b = colors.copy(), zt.copy()
    fg(c_b, z_b)
    got, _, _ = _fill_case(valid, z_b, c_b)
    assert np.array_equal(ref[v, L + 1 : R], got[v, L + 1 : R])
    # ...but one at exactly the occluder depth is not
    c_c, z_c = colors.copy(), zt.copy()
    z_c[1, 11] = 2.0
    c_d, z_d = c_c.copy(), z_c.copy()
    c_d[1, 11] = 255 - c_d[1, 11]
    o1, _, _ = _fill_case(valid, z_c, c_c)
    o2, _, _ = _fill_case(valid, z_d, c_d)
    assert not np.array_equal(o1[v, L + 1 : R], o2[v, L + 1 : R])


def test_fill_row_order_top_row_first():
    """Rows are visited v-1, v, v+1: the top-row contributor takes weight 1 - q of the total."""
    h, w = 3, 16
    valid = np.zeros((h, w), bool)
    valid[1, :4] = True   # L = 3 in the middle row
    valid[1, 6] = True    # R = 6, hole 4..5, width 3, kernel columns 9..6
    valid[0, 7] = True    # top-row contributor
    valid[2, 9] = True    # bottom-row contributor
    zt = np.where(valid, 5.0, np.inf)
    zt[1, 6] = 1.0        # make R itself foreground so only the two rows contribute
    zt[1, 3] = 2.0        # occluder
    colors = np.zeros((h, w, 4), np.uint8)
    colors[0, 7] = (200, 40, 10, 255)
    colors[2, 9] = (100, 120, 250, 255)
    out, _, _ = _fill_case(valid, zt, colors)
    # u = 5: t = 1/3 -> (171, 63, 79, 255); u = 4: t = 2/3 -> (177, 58, 65, 255)
    assert out[1, 5].tolist() == [171, 63, 79, 255]
    assert out[1, 4].tolist() == [177, 58, 65, 255]


def test_fill_fallbacks():
    w = 10
    colors = np.arange(w * 4, dtype=np.uint8).reshape(1, w, 4)
    # right border: no background edge -> copy of the left neighbour L
    valid = np.array([[1, 1, 1, 1, 1, 1, 0, 0, 0, 0]], bool)
    out, _, _ = _fill_case(valid, np.where(valid, 3.0, np.inf), colors)
    assert (out[0, 6:] == colors[0, 5]).all()
    # every candidate is foreground -> copy of R
    valid = np.array([[1, 1, 0, 0, 1, 1, 1, 1, 1, 1]], bool)
    zt = np.where(valid, 1.0, np.inf)
    zt[0, 1] = 5.0  # occluder farther than all candidates
    out, _, _ = _fill_case(valid, zt, colors)
    assert (out[0, 2:4] == colors[0, 4]).all()
    # no reached pixel in the row and no rows around it -> zeros
    valid = np.zeros((1, w), bool)
    out, _, _ = _fill_case(valid, np.full((1, w), np.inf), colors)
    assert not out.any()
    # left border hole (L = -1): d_occ = 0, so the background candidates all count
    valid = np.array([[0, 0, 1, 1, 1, 1, 1, 1, 1, 1]], bool)
    c2 = np.zeros((1, w, 4), np.uint8)
    c2[0, 2:] = (9, 8, 7, 6)
    out, _, _ = _fill_case(valid, np.where(valid, 0.5, np.inf), c2)
    assert (out[0, :2] == (9, 8, 7, 6)).all()


# ----------------------------------------------------------------------------- analytic ray-cast
def _near_silhouette(prim):
    p = np.pad(prim, 1, mode="edge")
    h, w = prim.shape
    m = np.zeros_like(prim, bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            m |= p[1 + dy : 1 + dy + h, 1 + dx : 1 + dx + w] != prim
    return m


def test_raycast_second_eye_agreement():
    """On tiny scenes, warped visible pixels show the primitive the true right eye sees.

    For right-eye pixels that are reached (not holes) and not within one pixel of a
    silhouette in either eye, the source pixel's primitive id must equal the ray-cast
    right-eye primitive id, and the warped depth must match the true depth within 1%.
    """
    agree = total = 0
    depth_ok = 0
    for seed in range(1, 21):
        cfg = scene.SceneConfig(w=64, h=64, n_prims=1 + seed % 4, ground=seed % 2 == 0,
                                log_depth=False, zmin=0.4, zmax=6.0, ipd=0.063)
        (cl, dl, pl), (cr, dr, pr) = scene.render_pair(cfg, seed)
        st = oracle.synthesize_steps(cl, dl, cfg.fx, cfg.ipd, cfg.near, cfg.far)
        src, zt = st["src"], st["zt"]
        sil_l, sil_r = _near_silhouette(pl), _near_silhouette(pr)
        for y in range(cfg.h):
            for u in range(cfg.w):
                s = src[y, u]
                if s < 0 or sil_r[y, u] or sil_l[y, s]:
                    continue
                total += 1
                agree += pl[y, s] == pr[y, u]
                if pr[y, u] >= 0:
                    depth_ok += abs(float(zt[y, u]) - float(dr[y, u])) <= 0.01 * float(dr[y, u])
                else:
                    depth_ok += 1
    assert total > 20000
    assert agree / total >= 0.995, agree / total
    assert depth_ok / total >= 0.99, depth_ok / total


def test_raycast_sign_of_motion():
    """A near object moves left (toward -x) in the right eye: pixels move in one direction (O1)."""
    cfg = scene.SceneConfig(w=128, h=64, n_prims=1, ground=False, log_depth=False, zmin=0.5,
                            zmax=0.6, ipd=0.063)
    (cl, dl, pl), (cr, dr, pr) = scene.render_pair(cfg, 5)
    st = oracle.synthesize_steps(cl, dl, cfg.fx, cfg.ipd, cfg.near, cfg.far)
    src = st["src"]
    ys, us = np.nonzero(src >= 0)
    assert (src[ys, us] >= us).all()  # every reached target comes from the same or a larger column
    cols_l = np.nonzero((pl == 0).any(axis=0))[0]
    cols_r = np.nonzero((pr == 0).any(axis=0))[0]
    assert cols_r.mean() < cols_l.mean()


# ----------------------------------------------------------------------------- whole path
@pytest.mark.parametrize("seed", [1, 2])
def test_whole_path_consistency(seed):
    """The one-call path equals the step-by-step path, and reached pixels copy their source."""
    cfg = scene.small_config()
    c, d, _ = scene.render(cfg, seed)
    out, mask = oracle.synthesize(c, d, cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.ipd, cfg.near, cfg.far)
    st = oracle.synthesize_steps(c, d, cfg.fx, cfg.ipd, cfg.near, cfg.far)
    assert np.array_equal(out, st["out"]) and np.array_equal(mask, st["mask"])
    src = st["src"]
    assert np.array_equal(mask, (src < 0).astype(np.uint8))
    ys, us = np.nonzero(src >= 0)
    assert np.array_equal(out[ys, us], c[ys, src[ys, us]])
    assert mask.any()


def test_empty_frame():
    out, mask = oracle.synthesize(np.zeros((0, 0, 4), np.uint8), np.zeros((0, 0), np.float32),
                                  1.0, 1.0, 0.0, 0.0, 0.063, 0.05, 1000.0)
    assert out.shape == (0, 0, 4) and mask.shape == (0, 0)
