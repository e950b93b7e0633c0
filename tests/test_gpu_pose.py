"""General second-eye pose (Eq. 5 with a general M) on the GPU, byte for byte against the
CPU oracle with the same pose (needs a GPU)."""
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


def _rot(yaw, pitch, roll):
    cy_, sy = np.cos(yaw), np.sin(yaw)
    cp, sp = np.cos(pitch), np.sin(pitch)
    cr, sr = np.cos(roll), np.sin(roll)
    ry = np.array([[cy_, 0, sy], [0, 1, 0], [-sy, 0, cy_]])
    rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    rz = np.array([[cr, -sr, 0], [sr, cr, 0], [0, 0, 1]])
    return (rz @ rx @ ry).astype(np.float32)


POSES = [(np.eye(3, dtype=np.float32), [0.063, 0.0, 0.0]),
         (_rot(0.02, 0.0, 0.0), [0.063, 0.0, 0.0]),
         (_rot(0.0, 0.03, 0.01), [0.063, 0.015, 0.0]),
         (_rot(-0.04, 0.02, -0.03), [0.05, -0.02, 0.04])]


def _run(y, c, d, cam, pose, kernel_rows=3, nearest_first=False, unfused=False):
    syn = y.Synthesizer(**cam, kernel_rows=kernel_rows, nearest_first=nearest_first, pose=pose)
    out, mask = syn(torch.from_numpy(np.ascontiguousarray(c)).to(DEV),
                    torch.from_numpy(np.ascontiguousarray(d)).to(DEV), unfused=unfused)
    torch.cuda.synchronize()
    assert syn.status() == 0
    syn.close()
    return out.cpu().numpy(), mask.cpu().numpy()


def _ref(c, d, cam, pose, kernel_rows=3, nearest_first=False):
    return oracle.synthesize_pose(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], pose[0], pose[1], cam["near"],
                                  cam["far"], kernel_rows=kernel_rows, nearest_first=nearest_first)


def _same(got, ref, what):
    bad = np.nonzero((got[0] != ref[0]).any(axis=-1) | (got[1] != ref[1]))
    assert bad[0].size == 0, f"{what}: {bad[0].size} pixels differ, first at {bad[0][0]},{bad[1][0]}"


@pytest.mark.parametrize("k", range(len(POSES)))
def test_small_scenes(yoro, k):
    cfg = scene.small_config()
    cam = cfg.camera()
    for seed in (1, 2):
        c, d, _ = scene.render(cfg, seed)
        ref = _ref(c, d, cam, POSES[k])
        _same(_run(yoro, c, d, cam, POSES[k]), ref, f"seed {seed} pose {k}")
        _same(_run(yoro, c, d, cam, POSES[k], unfused=True), ref, f"unfused call, seed {seed} pose {k}")


@pytest.mark.parametrize("k", (1, 3))
def test_quest_frame(yoro, k):
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 3)
    cam = cfg.camera()
    _same(_run(yoro, c, d, cam, POSES[k]), _ref(c, d, cam, POSES[k]), f"quest pose {k}")


def test_kernel_variant_and_dyadic_translation_equals_the_base_path(yoro):
    rng = np.random.default_rng(4)
    h, w = 40, 96
    d = rng.choice(np.array([0.5, 1.0, 2.0, 4.0], np.float32), (h, w // 4)).repeat(4, axis=1)
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    cam = dict(w=w, h=h, fx=32.0, fy=32.0, cx=48.0, cy=20.0, ipd=0.25, near=0.05, far=1000.0)
    base = oracle.synthesize(c, d, 32.0, 32.0, 48.0, 20.0, 0.25, 0.05, 1000.0, kernel_rows=5, nearest_first=True)
    got = _run(yoro, c, d, cam, (np.eye(3), [0.25, 0.0, 0.0]), kernel_rows=5, nearest_first=True)
    _same(got, base, "translation h 5 nearest-first")


def test_frame_too_wide_for_a_band(yoro):
    w, h = 9984, 6
    assert w > yoro.yoro_max_fused_width()
    rng = np.random.default_rng(8)
    d = np.repeat(rng.uniform(0.3, 6.0, (h, w // 8)).astype(np.float32), 8, axis=1)
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    cam = dict(w=w, h=h, fx=w / 2.0, fy=w / 2.0, cx=w / 2.0, cy=h / 2.0, ipd=0.0, near=0.05, far=1000.0)
    pose = POSES[2]
    _same(_run(yoro, c, d, cam, pose), _ref(c, d, cam, pose), "wide")


def test_host_and_mapped_entry_points_take_the_variant_paths(yoro):
    """yoro_synthesize_host and yoro_synthesize_mapped of a pose handle and of an
    intermediate-buffer handle give the oracle's result too."""
    cfg = scene.small_config()
    cam = cfg.camera()
    c, d, _ = scene.render(cfg, 5)
    cases = [(yoro.yoro_create_pose(cam["w"], cam["h"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], POSES[3][0],
                                    POSES[3][1], cam["near"], cam["far"]),
              _ref(c, d, cam, POSES[3])),
             (yoro.yoro_create_imb(**cam, imbuffer_div=4, interpolate=True),
              oracle.synthesize_imb(c, d, cam["fx"], cam["ipd"], cam["near"], cam["far"], 4, True))]
    for hdl, ref in cases:
        for fn in (yoro.yoro_synthesize_host, yoro.yoro_synthesize_mapped):
            hc = torch.from_numpy(c).pin_memory()
            hd = torch.from_numpy(d).pin_memory()
            ho = torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8).pin_memory()
            hm = torch.empty((cfg.h, cfg.w), dtype=torch.uint8).pin_memory()
            fn(hdl, hc, hd, ho, hm)
            torch.cuda.synchronize()
            assert yoro.yoro_stream_status(hdl) == 0
            _same((ho.numpy(), hm.numpy()), ref, fn.__name__)
        yoro.yoro_destroy(hdl)
