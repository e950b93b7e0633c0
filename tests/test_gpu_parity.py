"""CUDA path vs the CPU oracle, byte for byte, through the C ABI (needs a GPU).

The bar is bit-exact: the warp indices, the nearest-wins z-buffer and the RGBA8
output are integer results of binary32 arithmetic that both sides perform in the
same order, so the right eye and the hole mask must match exactly.
"""
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


def _ref(color, depth, cam):
    return oracle.synthesize(color, depth, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"], cam["near"],
                             cam["far"])


def _run(y, color, depth, cam, unfused=False, stream=None):
    syn = y.Synthesizer(**cam)
    out, mask = syn(torch.from_numpy(np.ascontiguousarray(color)).to(DEV),
                    torch.from_numpy(np.ascontiguousarray(depth)).to(DEV), stream=stream, unfused=unfused)
    torch.cuda.synchronize()
    assert syn.status(stream) == 0
    syn.close()
    return out.cpu().numpy(), mask.cpu().numpy()


def _assert_same(got, ref, what=""):
    go, gm = got
    ro, rm = ref
    bad_px = np.nonzero((go != ro).any(axis=-1) | (gm != rm))
    assert bad_px[0].size == 0, f"{what}: {bad_px[0].size} pixels differ, first at {bad_px[0][0]},{bad_px[1][0]}"


def _cam(w, h, fx=None, ipd=0.063, near=0.05, far=1000.0):
    fx = w / 2.0 if fx is None else fx
    return dict(w=w, h=h, fx=fx, fy=fx, cx=w / 2.0, cy=h / 2.0, ipd=ipd, near=near, far=far)


def _random_frame(h, w, seed, zlo=0.05, zhi=3.0, bad=True):
    rng = np.random.default_rng(seed)
    # piecewise-constant depth runs make real occlusions and wide holes
    d = np.empty((h, w), np.float32)
    for y in range(h):
        x = 0
        while x < w:
            run = int(rng.integers(1, 40))
            d[y, x : x + run] = rng.uniform(zlo, zhi)
            x += run
    d *= rng.uniform(0.98, 1.02, (h, w)).astype(np.float32)
    if bad:
        flat = d.reshape(-1)
        idx = rng.choice(flat.size, size=max(1, flat.size // 50), replace=False)
        special = np.array([0.0, -0.0, -1.0, np.nan, np.inf, -np.inf, 1e-6, 5e6, 1e-40], np.float32)
        special = np.append(special, np.array([0xFFC00000], np.uint32).view(np.float32))  # negative NaN
        flat[idx] = rng.choice(special, idx.size)
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    return c, d


@pytest.mark.parametrize("seed", range(1, 17))
def test_small_scene_bit_exact(yoro, seed):
    cfg = scene.small_config()
    c, d, _ = scene.render(cfg, seed)
    cam = cfg.camera()
    _assert_same(_run(yoro, c, d, cam), _ref(c, d, cam), f"small seed {seed}")


@pytest.mark.parametrize("seed", range(1, 9))
def test_quest_frame_bit_exact(yoro, seed):
    """The 1832x1920 workload in the launch configuration the benchmark times."""
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, seed)
    cam = cfg.camera()
    ref = _ref(c, d, cam)
    assert ref[1].mean() > 0.02  # the workload has real disocclusions
    _assert_same(_run(yoro, c, d, cam), ref, f"quest seed {seed}")


@pytest.mark.parametrize("seed", [1, 2])
def test_unfused_bit_exact(yoro, seed):
    cfg = scene.small_config()
    c, d, _ = scene.render(cfg, seed)
    cam = cfg.camera()
    _assert_same(_run(yoro, c, d, cam, unfused=True), _ref(c, d, cam), "unfused small")


def test_unfused_quest_bit_exact(yoro):
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 3)
    cam = cfg.camera()
    _assert_same(_run(yoro, c, d, cam, unfused=True), _ref(c, d, cam), "unfused quest")


@pytest.mark.parametrize("h,w", [(1, 1), (1, 7), (7, 1), (3, 5), (67, 253), (33, 129), (5, 128), (9, 132),
                                 (2, 1832), (41, 1830), (17, 260), (11, 545), (6, 2500), (3, 1000)])
def test_ragged_sizes_random_depth(yoro, h, w):
    """Sizes that are not multiples of the 32/128-pixel blocks or of 4; hostile depths."""
    c, d = _random_frame(h, w, seed=h * 7919 + w)
    cam = _cam(w, h, fx=max(w / 2.0, 8.0), ipd=0.1)
    ref = _ref(c, d, cam)
    _assert_same(_run(yoro, c, d, cam), ref, f"fused {h}x{w}")
    _assert_same(_run(yoro, c, d, cam, unfused=True), ref, f"unfused {h}x{w}")


@pytest.mark.parametrize("seed", range(4))
def test_wide_holes_random_depth(yoro, seed):
    """Near/far runs with disparities of hundreds of pixels: holes wider than 128-pixel blocks."""
    h, w = 24, 1024
    c, d = _random_frame(h, w, seed=100 + seed, zlo=0.06, zhi=50.0)
    cam = _cam(w, h, ipd=0.063)
    ref = _ref(c, d, cam)
    assert ref[1].mean() > 0.05
    _assert_same(_run(yoro, c, d, cam), ref, "wide holes")


@pytest.mark.parametrize("per_row", [100, 1832])
def test_target_columns_on_a_rounding_boundary(yoro, per_row):
    """Depths whose disparity k/z is n + 1/2 put x + 0.5 - k/z on an integer, where the
    fast estimate of the target column cannot decide the floor and the IEEE division
    must.  100 such pixels per row fit the kernel's short list of deferred pixels; whole
    rows overflow it and take the rescan of the window."""
    h, w = 40, 1832
    cam = _cam(w, h, ipd=0.063)
    k = float(np.float32(cam["fx"]) * np.float32(cam["ipd"]))
    rng = np.random.default_rng(per_row)
    c, d = _random_frame(h, w, seed=77, zlo=0.3, zhi=20.0, bad=False)
    for y in range(h):
        cols = rng.choice(w, size=per_row, replace=False)
        n = rng.integers(1, 120, per_row)
        d[y, cols] = (k / (n + 0.5)).astype(np.float32)
    ref = _ref(c, d, cam)
    _assert_same(_run(yoro, c, d, cam), ref, "fused")
    _assert_same(_run(yoro, c, d, cam, unfused=True), ref, "unfused")


@pytest.mark.parametrize("h,w", [(11000, 96), (5200, 768), (12000, 40)])
def test_tall_bands(yoro, h, w):
    """Narrow, tall frames give bands of more than 32 rows (several 32-row steps in the
    per-row hole pass and in the fill's row search), on both launch shapes (one CTA per
    SM, and two half-height CTAs per SM)."""
    c, d = _random_frame(h, w, seed=h + w, zlo=0.05, zhi=30.0)
    cam = _cam(w, h, fx=max(w / 2.0, 8.0), ipd=0.08)
    _assert_same(_run(yoro, c, d, cam), _ref(c, d, cam), f"fused {h}x{w}")


@pytest.mark.parametrize("fx,ipd,near,far", [(916.0, 0.063, 1e-4, 1000.0), (916.0, 0.5, 0.05, 2.0),
                                             (5000.0, 0.063, 0.05, 1000.0), (916.0, 1e-6, 0.05, 1000.0)])
def test_extreme_cameras(yoro, fx, ipd, near, far):
    """Disparities up to millions of pixels (tiny near plane: every estimate undecided, the
    IEEE division decides all of them), a near far plane that clamps most depths, a long
    focal length, and a sub-pixel baseline."""
    h, w = 48, 1832
    c, d = _random_frame(h, w, seed=int(fx) + int(ipd * 1e3), zlo=0.01, zhi=50.0)
    cam = dict(w=w, h=h, fx=fx, fy=fx, cx=w / 2.0, cy=h / 2.0, ipd=ipd, near=near, far=far)
    ref = _ref(c, d, cam)
    _assert_same(_run(yoro, c, d, cam), ref, "fused")
    _assert_same(_run(yoro, c, d, cam, unfused=True), ref, "unfused")


def test_misaligned_pointers_take_the_element_path(yoro):
    h, w = 40, 96
    c, d = _random_frame(h, w, seed=5)
    cam = _cam(w, h, ipd=0.08)
    ref = _ref(c, d, cam)
    # views that start 4 bytes into their storage: 4-aligned, not 16-aligned
    cb = torch.zeros(h * w * 4 + 4, dtype=torch.uint8, device=DEV)
    cb[4:].copy_(torch.from_numpy(c).reshape(-1).to(DEV))
    db = torch.zeros(h * w + 1, dtype=torch.float32, device=DEV)
    db[1:].copy_(torch.from_numpy(d).reshape(-1).to(DEV))
    ob = torch.zeros(h * w * 4 + 4, dtype=torch.uint8, device=DEV)
    mb = torch.zeros(h * w + 1, dtype=torch.uint8, device=DEV)
    hdl = yoro.yoro_create(**cam)
    yoro.yoro_synthesize(hdl, cb[4:].view(h, w, 4), db[1:].view(h, w), ob[4:].view(h, w, 4), mb[1:].view(h, w))
    torch.cuda.synchronize()
    assert yoro.yoro_stream_status(hdl) == 0
    yoro.yoro_destroy(hdl)
    _assert_same((ob[4:].view(h, w, 4).cpu().numpy(), mb[1:].view(h, w).cpu().numpy()), ref, "misaligned")


def test_odd_address_is_rejected(yoro):
    h, w = 4, 8
    hdl = yoro.yoro_create(**_cam(w, h))
    lib = yoro.load_library()
    cb = torch.zeros(h * w * 4 + 1, dtype=torch.uint8, device=DEV)
    d = torch.ones(h, w, device=DEV)
    o = torch.zeros(h, w, 4, dtype=torch.uint8, device=DEV)
    m = torch.zeros(h, w, dtype=torch.uint8, device=DEV)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.yoro_synthesize(hdl.ptr, cb.data_ptr() + 1, d.data_ptr(), o.data_ptr(), m.data_ptr(), s) == 2
    # outputs aliasing inputs
    assert lib.yoro_synthesize(hdl.ptr, o.data_ptr(), d.data_ptr(), o.data_ptr(), m.data_ptr(), s) == 1
    assert lib.yoro_synthesize(hdl.ptr, None, d.data_ptr(), o.data_ptr(), m.data_ptr(), s) == 1
    yoro.yoro_destroy(hdl)


def test_ipd_zero_identity(yoro):
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 1)
    cam = dict(cfg.camera(), ipd=0.0)
    out, mask = _run(yoro, c, d, cam)
    assert np.array_equal(out, c) and not mask.any()


def test_max_fused_width_and_beyond(yoro):
    wmax = yoro.yoro_max_fused_width()
    assert wmax >= 2064  # every per-eye size of the workloads fits the fused kernel
    for w in (wmax, wmax + 4, wmax + 3):
        h = 6
        c, d = _random_frame(h, w, seed=w, zlo=0.2, zhi=20.0)
        cam = _cam(w, h)
        _assert_same(_run(yoro, c, d, cam), _ref(c, d, cam), f"width {w}")


def test_widths_around_the_scatter_column_split(yoro):
    """The scatter's two forms: whole columns per thread (x and x + 1024) where they
    split evenly enough over the 1024 threads, pixels dealt round-robin elsewhere and
    past column 2048: widths on either side of each switch."""
    for w in (800, 820, 1023, 1024, 1025, 1638, 1639, 2047, 2048, 2049, 2100, 2300):
        h = 29
        c, d = _random_frame(h, w, seed=w + 7, zlo=0.1, zhi=10.0)
        cam = _cam(w, h, ipd=0.08)
        _assert_same(_run(yoro, c, d, cam), _ref(c, d, cam), f"width {w}")


def _crack_frame(h, w, seed):
    """Rows of one-pixel cracks: even columns at disparity D, odd ones at D - 1, so every
    second target pixel is a crack (over the whole row, its left or its right part, or
    nowhere), with the rows' crack counts odd and even so that cracks dealt two per lane
    cross row ends."""
    rng = np.random.default_rng(seed)
    fx = w / 2.0
    cam = _cam(w, h, fx=fx, ipd=0.08)
    k = np.float32(fx) * np.float32(cam["ipd"])
    d = np.empty((h, w), np.float32)
    for y in range(h):
        dd = rng.uniform(3.2, 9.7)
        row = np.full(w, k / dd, np.float32)
        kind = y % 4
        if kind == 1:
            row[1::2] = k / (dd - 1.0)
        elif kind == 2:
            row[1 : int(rng.integers(w // 4, 3 * w // 4)) : 2] = k / (dd - 1.0)
        elif kind == 3:
            row[int(rng.integers(w // 4, 3 * w // 4)) | 1 :: 2] = k / (dd - 1.0)
        d[y] = row
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    return c, d, cam


def test_crack_dense_frames(yoro):
    """Thousands of one-pixel cracks per band (the fill deals them two per lane), single
    frames and one batched launch, byte for byte against the oracle."""
    frames, refs = [], []
    for h, w, seed in ((41, 301, 1), (64, 1832, 2), (29, 1024, 3)):
        c, d, cam = _crack_frame(h, w, seed)
        ref = _ref(c, d, cam)
        assert int(ref[1].sum()) > h * w // 5  # mostly cracks
        _assert_same(_run(yoro, c, d, cam), ref, f"cracks {w}x{h}")
        refs.append(ref)
        frames.append(dict(cam, color=torch.from_numpy(c).to(DEV), depth=torch.from_numpy(d).to(DEV),
                           out_color=torch.empty((h, w, 4), dtype=torch.uint8, device=DEV),
                           out_mask=torch.empty((h, w), dtype=torch.uint8, device=DEV)))
    yoro.yoro_synthesize_batch(frames)
    torch.cuda.synchronize()
    assert yoro.yoro_stream_status(None) == 0
    for fr, ref in zip(frames, refs):
        _assert_same((fr["out_color"].cpu().numpy(), fr["out_mask"].cpu().numpy()), ref, f"batch cracks {fr['w']}")


def test_empty_frames(yoro):
    for w, h in ((0, 0), (0, 5), (5, 0)):
        hdl = yoro.yoro_create(**_cam(max(w, 1), h) | dict(w=w, h=h))
        lib = yoro.load_library()
        assert lib.yoro_synthesize(hdl.ptr, None, None, None, None, None) == 0
        yoro.yoro_destroy(hdl)


def test_host_api_matches(yoro):
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 2)
    cam = cfg.camera()
    hdl = yoro.yoro_create(**cam)
    hc = torch.from_numpy(c).pin_memory()
    hd = torch.from_numpy(d).pin_memory()
    ho = torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8).pin_memory()
    hm = torch.empty((cfg.h, cfg.w), dtype=torch.uint8).pin_memory()
    for _ in range(2):
        yoro.yoro_synthesize_host(hdl, hc, hd, ho, hm)
        torch.cuda.synchronize()
        _assert_same((ho.numpy(), hm.numpy()), _ref(c, d, cam), "host api")
    assert yoro.yoro_stream_status(hdl) == 0
    yoro.yoro_destroy(hdl)


def test_mapped_host_buffers(yoro):
    """Zero copy: the kernels read and write page-locked host memory directly; pageable
    host memory and device memory are refused before any launch."""
    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 5)
    cam = cfg.camera()
    hdl = yoro.yoro_create(**cam)
    hc = torch.from_numpy(c).pin_memory()
    hd = torch.from_numpy(d).pin_memory()
    ho = torch.zeros((cfg.h, cfg.w, 4), dtype=torch.uint8).pin_memory()
    hm = torch.zeros((cfg.h, cfg.w), dtype=torch.uint8).pin_memory()
    yoro.yoro_synthesize_mapped(hdl, hc, hd, ho, hm)
    torch.cuda.synchronize()
    _assert_same((ho.numpy(), hm.numpy()), _ref(c, d, cam), "mapped")
    lib = yoro.load_library()
    pageable = torch.from_numpy(c.copy())
    assert lib.yoro_synthesize_mapped(hdl.ptr, pageable.data_ptr(), hd.data_ptr(), ho.data_ptr(), hm.data_ptr(),
                                      None) == 1
    dev = torch.from_numpy(d).to(DEV)
    assert lib.yoro_synthesize_mapped(hdl.ptr, hc.data_ptr(), dev.data_ptr(), ho.data_ptr(), hm.data_ptr(),
                                      None) == 1
    yoro.yoro_destroy(hdl)


def test_side_stream_and_two_handles(yoro):
    cfg = scene.small_config()
    s = torch.cuda.Stream()
    frames = [scene.render(cfg, seed)[:2] for seed in (3, 4)]
    cam = cfg.camera()
    outs = []
    syns = [yoro.Synthesizer(**cam), yoro.Synthesizer(**dict(cam, ipd=0.07))]
    with torch.cuda.stream(s):
        for syn, (c, d) in zip(syns, frames):
            outs.append(syn(torch.from_numpy(c).to(DEV), torch.from_numpy(d).to(DEV), stream=s))
    s.synchronize()
    for (c, d), (o, m), ipd in zip(frames, outs, (cfg.ipd, 0.07)):
        _assert_same((o.cpu().numpy(), m.cpu().numpy()), _ref(c, d, dict(cam, ipd=ipd)), "side stream")
    for syn in syns:
        assert syn.status(s) == 0
        syn.close()


def test_batch_mixed_sizes(yoro):
    """One persistent launch over frames of different sizes and cameras equals per-frame results."""
    specs = [(scene.SceneConfig(w=w, h=h, n_prims=60, ground=True, log_depth=True, zmin=0.1, zmax=100.0,
                                ipd=ipd), seed)
             for (w, h), ipd, seed in zip([(1024, 1024), (1440, 1600), (1832, 1920), (2064, 2208), (256, 256)],
                                          [0.055, 0.072, 0.063, 0.06, 0.063], [11, 12, 13, 14, 15])]
    frames, refs = [], []
    for cfg, seed in specs:
        c, d, _ = scene.render(cfg, seed)
        refs.append(_ref(c, d, cfg.camera()))
        frames.append(dict(cfg.camera(), color=torch.from_numpy(c).to(DEV), depth=torch.from_numpy(d).to(DEV),
                           out_color=torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8, device=DEV),
                           out_mask=torch.empty((cfg.h, cfg.w), dtype=torch.uint8, device=DEV)))
    # a ragged frame travels in the same launch
    c, d = _random_frame(37, 301, seed=9)
    cam = _cam(301, 37, ipd=0.1)
    refs.append(_ref(c, d, cam))
    frames.append(dict(cam, color=torch.from_numpy(c).to(DEV), depth=torch.from_numpy(d).to(DEV),
                       out_color=torch.empty((37, 301, 4), dtype=torch.uint8, device=DEV),
                       out_mask=torch.empty((37, 301), dtype=torch.uint8, device=DEV)))
    yoro.yoro_synthesize_batch(frames)
    torch.cuda.synchronize()
    assert yoro.yoro_stream_status(None) == 0
    for fr, ref in zip(frames, refs):
        _assert_same((fr["out_color"].cpu().numpy(), fr["out_mask"].cpu().numpy()), ref, f"batch {fr['w']}")
