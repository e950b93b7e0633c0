"""The row-downsampled intermediate buffer (strategies (c) and (d)) on the GPU, byte
for byte against the CPU oracle with the same cells and interpolation (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_15183_gb300 import scene

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def yoro():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_15183_gb300 as y
    from paper_2506_15183_gb300 import _build

    _build.build_cuda()
    oracle.build()
    scene.build()
    y.load_library()
    return y


def _run(y, c, d, cam, div, interp, kernel_rows=3, nearest_first=False, unfused=False):
    syn = y.Synthesizer(**cam, kernel_rows=kernel_rows, nearest_first=nearest_first, imbuffer_div=div,
                        interpolate=interp)
    out, mask = syn(torch.from_numpy(np.ascontiguousarray(c)).to(DEV),
                    torch.from_numpy(np.ascontiguousarray(d)).to(DEV), unfused=unfused)
    torch.cuda.synchronize()
    assert syn.status() == 0
    syn.close()
    return out.cpu().numpy(), mask.cpu().numpy()


def _ref(c, d, cam, div, interp, kernel_rows=3, nearest_first=False):
    return oracle.synthesize_imb(c, d, cam["fx"], cam["ipd"], cam["near"], cam["far"], div, interp,
                                 kernel_rows=kernel_rows, nearest_first=nearest_first)


def _same(got, ref, what):
    bad = np.nonzero((got[0] != ref[0]).any(axis=-1) | (got[1] != ref[1]))
    assert bad[0].size == 0, f"{what}: {bad[0].size} pixels differ, first at {bad[0][0]},{bad[1][0]}"


@pytest.mark.parametrize("div", (1, 2, 4, 8, 16))
@pytest.mark.parametrize("interp", (False, True))
def test_small_scenes(yoro, div, interp):
    cfg = scene.small_config()
    cam = cfg.camera()
    for seed in (1, 2):
        c, d, _ = scene.render(cfg, seed)
        ref = _ref(c, d, cam, div, interp)
        _same(_run(yoro, c, d, cam, div, interp), ref, f"seed {seed} div {div} interp {interp}")
        # the separate kernels (cells, sampling, band fill over the sampled image)
        _same(_run(yoro, c, d, cam, div, interp, unfused=True), ref, f"unfused call, seed {seed}")


def test_one_cell_per_pixel_is_the_base_path(yoro):
    cfg = scene.small_config()
    cam = cfg.camera()
    c, d, _ = scene.render(cfg, 3)
    ref = oracle.synthesize(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"], cam["near"], cam["far"])
    _same(_run(yoro, c, d, cam, 1, False), ref, "div 1")


@pytest.mark.parametrize("div,interp", [(2, False), (4, True), (16, True)])
def test_quest_frame(yoro, div, interp):
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 2)
    cam = cfg.camera()
    _same(_run(yoro, c, d, cam, div, interp), _ref(c, d, cam, div, interp), f"quest div {div} interp {interp}")


def test_kernel_variant_with_cells(yoro):
    cfg = scene.small_config()
    cam = cfg.camera()
    c, d, _ = scene.render(cfg, 4)
    ref = _ref(c, d, cam, 4, True, kernel_rows=5, nearest_first=True)
    _same(_run(yoro, c, d, cam, 4, True, kernel_rows=5, nearest_first=True), ref, "h 5 nearest-first")


@pytest.mark.parametrize("w", (1, 7, 33, 1000))
def test_ragged_widths_and_extreme_cameras(yoro, w):
    rng = np.random.default_rng(w)
    h = 21
    d = np.repeat(rng.uniform(0.05, 8.0, (h, (w + 4) // 5)).astype(np.float32), 5, axis=1)[:, :w].copy()
    d[rng.random((h, w)) < 0.02] = np.nan  # invalid depths take far
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    for fx, ipd in ((w / 2.0, 0.063), (5000.0, 2.0), (w / 2.0, 0.0)):
        cam = dict(w=w, h=h, fx=fx, fy=fx, cx=w / 2.0, cy=h / 2.0, ipd=ipd, near=0.05, far=1000.0)
        for div, interp in ((2, True), (16, False), (8, True)):
            _same(_run(yoro, c, d, cam, div, interp), _ref(c, d, cam, div, interp),
                  f"w {w} fx {fx} ipd {ipd} div {div} interp {interp}")


def test_frame_too_wide_for_a_band(yoro):
    """Wider than any band window: the separate kernels with the per-pixel fill."""
    w, h = 9984, 5
    assert w > yoro.yoro_max_fused_width()
    rng = np.random.default_rng(99)
    d = np.repeat(rng.uniform(0.05, 6.0, (h, w // 8)).astype(np.float32), 8, axis=1)
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    cam = dict(w=w, h=h, fx=w / 2.0, fy=w / 2.0, cx=w / 2.0, cy=h / 2.0, ipd=0.063, near=0.05, far=1000.0)
    for div, interp in ((4, True), (2, False)):
        ref = _ref(c, d, cam, div, interp)
        _same(_run(yoro, c, d, cam, div, interp), ref, f"wide div {div}")
        _same(_run(yoro, c, d, cam, div, interp, unfused=True), ref, f"wide unfused div {div}")
