"""The Patcher's variants (Sec. Patcher: kernel height h, column order) on the GPU,
byte for byte against the CPU oracle with the same variant (needs a GPU)."""
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
    y.load_library()
    return y


def _run(y, c, d, cam, kernel_rows, nearest_first, unfused=False):
    syn = y.Synthesizer(**cam, kernel_rows=kernel_rows, nearest_first=nearest_first)
    out, mask = syn(torch.from_numpy(c).to(DEV), torch.from_numpy(d).to(DEV), unfused=unfused)
    torch.cuda.synchronize()
    assert syn.status() == 0
    syn.close()
    return out.cpu().numpy(), mask.cpu().numpy()


def _ref(c, d, cam, kernel_rows, nearest_first):
    return oracle.synthesize(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"], cam["near"], cam["far"],
                             kernel_rows=kernel_rows, nearest_first=nearest_first)


def _same(got, ref, what):
    bad = np.nonzero((got[0] != ref[0]).any(axis=-1) | (got[1] != ref[1]))
    assert bad[0].size == 0, f"{what}: {bad[0].size} pixels differ, first at {bad[0][0]},{bad[1][0]}"


@pytest.mark.parametrize("kernel_rows,nearest_first", [(3, True), (1, False), (1, True), (5, False), (7, True),
                                                      (15, False)])
def test_quest_frame_variants(yoro, kernel_rows, nearest_first):
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 4)
    cam = cfg.camera()
    ref = _ref(c, d, cam, kernel_rows, nearest_first)
    base = _ref(c, d, cam, 3, False)
    assert (ref[0] != base[0]).any()  # the variant changes the fill on this frame
    _same(_run(yoro, c, d, cam, kernel_rows, nearest_first), ref, f"fused h={kernel_rows} nf={nearest_first}")


@pytest.mark.parametrize("kernel_rows,nearest_first", [(1, True), (5, False), (9, True)])
def test_small_scenes_variants_fused_and_unfused(yoro, kernel_rows, nearest_first):
    cfg = scene.small_config()
    for seed in (1, 2, 3):
        c, d, _ = scene.render(cfg, seed)
        cam = cfg.camera()
        ref = _ref(c, d, cam, kernel_rows, nearest_first)
        _same(_run(yoro, c, d, cam, kernel_rows, nearest_first), ref, f"fused seed {seed}")
        _same(_run(yoro, c, d, cam, kernel_rows, nearest_first, unfused=True), ref, f"unfused seed {seed}")


def test_variant_on_tall_narrow_bands(yoro):
    """Bands of more than 32 rows with a 7-row kernel (3 halo rows on each side)."""
    rng = np.random.default_rng(5)
    h, w = 9000, 64
    d = np.repeat(rng.uniform(0.05, 20.0, (h, w // 8)).astype(np.float32), 8, axis=1)
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    cam = dict(w=w, h=h, fx=32.0, fy=32.0, cx=32.0, cy=h / 2.0, ipd=0.1, near=0.05, far=1000.0)
    ref = _ref(c, d, cam, 7, True)
    _same(_run(yoro, c, d, cam, 7, True), ref, "tall h=7 nearest-first")


def test_bad_options_are_rejected(yoro):
    cam = scene.small_config().camera()
    for kr, nf in ((2, False), (0, False), (17, False)):
        with pytest.raises(yoro.YoroError):
            yoro.yoro_create_ex(**cam, kernel_rows=kr, nearest_first=nf)
