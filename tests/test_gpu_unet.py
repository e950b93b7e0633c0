"""Tensor-core layers of the learned inpainter against its CPU definition (oracle/unet.py),
through the C ABI (needs a GPU).

A tcgen05 convolution sums the BF16 products in another order than the definition
(input channel, kernel row, kernel column), so the two agree within the error bound of
FP32 summation, not bit for bit.  For an output whose products are p_i (exact in FP32:
a product of two bfloat16 values has at most 16 significant bits), the definition's
sequential sum is within K u sum |p_i| of the exact sum (u = 2^-24, K products); the
tensor core's accumulation is allowed twice that (one unit in the last place per
addition).  So before rounding |gpu - oracle| <= 3 K u sum |p_i| + the bias addition's
rounding; after ReLU and rounding to bfloat16 the two may also land one bfloat16 step
apart where the value sits next to a rounding boundary.  The test allows exactly that
per element: tol = 3 K u sum|p| (1 + 2^-7) + 2 ulp_f32(|o|) + ulp_bf16(max(|o|, |g|)).
"""
import numpy as np
import pytest
import torch

from oracle import unet as ref

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def un():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_15183_gb300 as yoro
    from paper_2506_15183_gb300 import _build
    from paper_2506_15183_gb300 import unet

    _build.build_cuda()
    yoro.load_library()
    return unet


def _bf16_t(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()


def _ulp_bf16(v):
    v = np.maximum(np.abs(v), np.float32(2.0 ** -126))
    return np.exp2(np.floor(np.log2(v)) - 7).astype(np.float64)


def _case(un, T, H, W, cin, cout, seed, upsample=False, cy=None, coff=0, relu=True, real_cin=None):
    rng = np.random.default_rng(seed)
    real_cin = real_cin or cin
    x = np.zeros((T, real_cin, H, W), np.float32)
    x[:] = ref.bf16(rng.uniform(0.0, 1.0, x.shape).astype(np.float32))
    w = ref.bf16(rng.normal(0.0, np.sqrt(2.0 / (9 * real_cin)), (cout, real_cin, 3, 3)).astype(np.float32))
    b = rng.normal(0.0, 0.05, cout).astype(np.float32)
    # GPU: NHWC with Cin padded to a multiple of 32
    xp = np.zeros((T, H, W, cin), np.float32)
    xp[..., :real_cin] = np.transpose(x, (0, 2, 3, 1))
    cy = cy or cout
    f = 2 if upsample else 1
    y = torch.full((T, f * H, f * W, cy), 7.0, dtype=torch.bfloat16, device="cuda")
    wk = un.kmajor(w)
    if wk.shape[1] != 9 * cin:
        wk2 = np.zeros((cout, 9 * cin), np.float32)
        wk3 = wk.reshape(cout, 9, -1)
        wk2.reshape(cout, 9, cin)[:, :, :wk3.shape[2]] = wk3
        wk = wk2
    un.conv3x3(_bf16_t(xp), _bf16_t(wk), torch.from_numpy(b).cuda(), y, y_coff=coff, upsample=upsample, relu=relu)
    assert un.status() == 0
    g = y.float().cpu().numpy()
    for t in range(T):
        pre = ref.conv3x3(x[t], w, b)
        o = ref.relu_bf16(pre) if relu else ref.bf16(pre)
        absum = ref.conv3x3(np.abs(x[t]), np.abs(w), np.zeros(cout, np.float32)).astype(np.float64)
        K = 9 * real_cin
        go = g[t][..., coff:coff + cout]
        if upsample:
            for a in (0, 1):
                for c in (0, 1):
                    _compare(go[a::2, c::2].transpose(2, 0, 1), o, absum, K)
        else:
            _compare(go.transpose(2, 0, 1), o, absum, K)
        # channels outside [coff, coff + cout) are untouched
        if cy > cout:
            rest = np.delete(g[t], np.arange(coff, coff + cout), axis=-1)
            assert np.all(rest == 7.0)


def _compare(g, o, absum, K):
    o64, g64 = o.astype(np.float64), g.astype(np.float64)
    tol = 3 * K * U * absum * (1 + 2.0 ** -7) + 2 * np.abs(o64) * 2.0 ** -23 + _ulp_bf16(np.maximum(np.abs(o), np.abs(g)))
    bad = np.abs(g64 - o64) > tol
    assert not bad.any(), f"{bad.sum()} of {bad.size} outside the bound; worst {np.abs(g64 - o64)[bad].max()}"
    assert np.mean(g64 != o64) < 0.05  # almost every element is the same bfloat16 value


@pytest.mark.parametrize("T,H,W,cin,cout", [(1, 64, 64, 32, 32), (2, 32, 32, 32, 64), (1, 16, 16, 64, 128),
                                              (2, 8, 8, 128, 256), (3, 16, 16, 384, 128), (1, 64, 64, 96, 32)])
def test_conv_layer_matches_definition(un, T, H, W, cin, cout):
    _case(un, T, H, W, cin, cout, seed=100 + cin + cout)


@pytest.mark.parametrize("T,H,W,cin,cout", [(1, 64, 128, 32, 32), (2, 8, 64, 64, 32), (1, 32, 16, 64, 128),
                                              (1, 6, 64, 32, 32), (3, 16, 32, 32, 64)])
def test_conv_row_bands(un, T, H, W, cin, cout):
    """Both forms of the convolution: several row bands per image (whole-row halo boxes,
    rows -1 and H outside the image read as zeros, W = 128 boxes), and heights that no band
    of 256 pixels divides (the one-tile form)."""
    _case(un, T, H, W, cin, cout, seed=200 + H + W + cin + cout)


def test_conv_first_layer_padded_channels(un):
    """The 6 input channels padded to 32 with zero channels and zero weights."""
    _case(un, 1, 64, 64, 32, 32, seed=7, real_cin=6)


def test_conv_into_concat_buffer_and_upsampled(un):
    """Channel offset inside a wider buffer, and the 2x2 nearest-upsampling store."""
    _case(un, 2, 8, 8, 256, 256, seed=8, upsample=True, cy=384, coff=128)
    _case(un, 1, 32, 32, 64, 32, seed=9, cy=96, coff=0)
    _case(un, 1, 32, 32, 64, 64, seed=11, upsample=True, cy=96, coff=32)
    _case(un, 2, 16, 16, 128, 128, seed=12, upsample=True, cy=192, coff=64)


def test_conv_without_relu(un):
    _case(un, 1, 16, 16, 64, 64, seed=10, relu=False)


# ---- the whole network and the frame path -------------------------------------------

def _frame_tiles(seed, w=256, h=256):
    """A plain-path frame of a small scene (oracle steps) and its 64x64 tile inputs."""
    import oracle
    from paper_2506_15183_gb300 import scene

    cfg = scene.small_config().replace(w=w, h=h)
    c, d, _ = scene.render(cfg, seed)
    st = oracle.synthesize_steps(c, d, cfg.fx, cfg.ipd, cfg.near, cfg.far)
    return cfg, c, d, st


def _pad_to_tiles(a, h, w):
    H, W = (h + 63) // 64 * 64, (w + 63) // 64 * 64
    out = np.zeros((H, W) + a.shape[2:], a.dtype)
    out[:h, :w] = a
    return out


def _weights(seed):
    p = ref.init_weights(seed)
    rng = np.random.default_rng(seed + 1)
    for name, _, bs in ref.layer_shapes():
        p[name + ".b"] = rng.normal(0.0, 0.05, bs).astype(np.float32)
    return p


def _x_gpu(xs):
    """(T, 6, 64, 64) definition inputs -> (T, 64, 64, 32) bf16 on the GPU."""
    T = xs.shape[0]
    x = np.zeros((T, 64, 64, 32), np.float32)
    x[..., :6] = np.transpose(xs, (0, 2, 3, 1))
    return _bf16_t(x)


def _net(un, p, **kw):
    names = [n for n, _, _ in ref.layer_shapes()]
    return un.Inpainter(un.flatten_params(p, names), **kw)


def test_forward_matches_definition(un):
    """The 14 tensor-core layers, pools, upsampled concatenations and the output layer
    on three tiles of a warped frame (an odd count: the 8 x 8 level pairs tiles).  The
    layers agree with the definition within their bound (test above); through the
    network those one-step bfloat16 differences propagate, so the colors are compared
    with a sanity bound: every color within 0.03, mean within 0.003 (of [0, 1])."""
    cfg, c, d, st = _frame_tiles(3)
    hole_tiles = [(ty, tx) for ty in range(4) for tx in range(4)
                  if st["mask"][64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64].any()][:3]
    assert len(hole_tiles) == 3
    xs = np.stack([ref.tile_input(st["out"][64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64],
                                  st["mask"][64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64],
                                  st["zt"][64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64],
                                  d[64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64], cfg.near)
                   for ty, tx in hole_tiles])
    p = _weights(11)
    net = _net(un, p, max_tiles=4)
    rgb = torch.zeros((3, 64, 64, 3), dtype=torch.float32, device="cuda")
    net.forward(_x_gpu(xs), rgb)
    assert un.status() == 0
    g = rgb.cpu().numpy()
    for t in range(3):
        o = ref.forward(xs[t], p).transpose(1, 2, 0)
        diff = np.abs(g[t].astype(np.float64) - o)
        assert diff.max() <= 0.03 and diff.mean() <= 0.003, (t, diff.max(), diff.mean())
    net.close()


def test_every_layer_on_the_definitions_activations(un):
    """Each layer of a real forward pass, fed the definition's own input for that layer
    (so no earlier difference propagates), against the definition's output, within the
    per-layer bound of the tests above: real weights and activations, the skip
    concatenations and the upsampled stores."""
    cfg, c, d, st = _frame_tiles(4)
    ty, tx = next((ty, tx) for ty in range(4) for tx in range(4)
                  if st["mask"][64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64].any())
    sl = np.s_[64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64]
    x = ref.bf16(ref.tile_input(st["out"][sl], st["mask"][sl], st["zt"][sl], d[sl], cfg.near))
    p = {k: (ref.bf16(v) if k.endswith(".w") else v) for k, v in _weights(12).items()}
    layers = []  # (name, input (C, H, W), output (C, H, W))
    a, skips = x, []
    for l in range(4):
        if l:
            a = ref.maxpool2(a)
        for s in "ab":
            o = ref.relu_bf16(ref.conv3x3(a, p[f"enc{l}{s}.w"], p[f"enc{l}{s}.b"]))
            layers.append((f"enc{l}{s}", a, o))
            a = o
        skips.append(a)
    for l in (2, 1, 0):
        a = np.concatenate([skips[l], ref.upsample2(a)], axis=0)
        for s in "ab":
            o = ref.relu_bf16(ref.conv3x3(a, p[f"dec{l}{s}.w"], p[f"dec{l}{s}.b"]))
            layers.append((f"dec{l}{s}", a, o))
            a = o
    for name, xin, o in layers:
        cin, H, W = xin.shape
        cp = un.pad32(cin)
        xg = np.zeros((2, H, W, cp), np.float32)  # two copies: the 8 x 8 level takes tiles in pairs
        xg[:, :, :, :cin] = np.transpose(xin, (1, 2, 0))[None]
        w = p[name + ".w"]
        cout = w.shape[0]
        y = torch.zeros((2, H, W, cout), dtype=torch.bfloat16, device="cuda")
        un.conv3x3(_bf16_t(xg), _bf16_t(un.kmajor(w)), torch.from_numpy(p[name + ".b"]).cuda(), y)
        assert un.status() == 0
        absum = ref.conv3x3(np.abs(xin), np.abs(w), np.zeros(cout, np.float32)).astype(np.float64)
        for t in range(2):
            _compare(y[t].float().cpu().numpy().transpose(2, 0, 1), o, absum, 9 * cin)


@pytest.mark.parametrize("w,h", [(256, 256), (200, 136)])
def test_inpaint_frame(un, w, h):
    """The frame path: hole cells found on the device, the last column's and row's windows
    shifted inward to the frame's edge, hole pixels of each cell composed from the
    network's colors, everything else untouched.
    Against the definition's compose() on the same tiles: reached pixels and hole-free
    tiles byte for byte; hole pixels within 8 levels, mean within 1 level."""
    import paper_2506_15183_gb300 as yoro

    cfg, c, d, st = _frame_tiles(5, w, h)
    syn = yoro.Synthesizer(**cfg.camera())
    hdl = syn.handle
    rgba = torch.empty((h, w, 4), dtype=torch.uint8, device="cuda")
    mask = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    zt = torch.empty((h, w), dtype=torch.float32, device="cuda")
    dg = torch.from_numpy(d).cuda()
    yoro.yoro_synthesize_zt(hdl, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
    torch.cuda.synchronize()
    plain = rgba.cpu().numpy()
    assert np.array_equal(plain, st["out"]) and np.array_equal(mask.cpu().numpy(), st["mask"])
    # the warped depth: the winner's clamped depth at reached pixels (Alg. 2's stored depth), 0 at holes
    assert np.array_equal(zt.cpu().numpy(), np.where(st["mask"].astype(bool), 0.0, st["zt"]).astype(np.float32))
    p = _weights(13)
    net = _net(un, p, max_w=w, max_h=h)
    net.inpaint(rgba, mask, zt, dg, cfg.near)
    assert un.status() == 0
    got = rgba.cpu().numpy()
    # the definition on each hole cell's window: the cell, or for the last column and row
    # the 64 x 64 window ending at the frame's edge; only the cell's pixels are written
    expect = plain.copy()
    for ty in range((h + 63) // 64):
        for tx in range((w + 63) // 64):
            cell = np.s_[64 * ty:64 * ty + 64, 64 * tx:64 * tx + 64]
            if not st["mask"][cell].any():
                continue
            y0, x0 = min(64 * ty, h - 64), min(64 * tx, w - 64)
            win = np.s_[y0:y0 + 64, x0:x0 + 64]
            col = ref.forward(ref.tile_input(st["out"][win], st["mask"][win], st["zt"][win], d[win], cfg.near), p)
            comp = ref.compose(plain[win], st["mask"][win], col)
            expect[cell] = comp[64 * ty - y0:64 * ty - y0 + 64, 64 * tx - x0:64 * tx - x0 + 64][
                :expect[cell].shape[0], :expect[cell].shape[1]]
    hole = st["mask"].astype(bool)
    assert np.array_equal(got[~hole], plain[~hole])
    diff = np.abs(got[hole].astype(int) - expect[hole].astype(int))
    assert diff.max() <= 8 and diff.mean() <= 1.0, (diff.max(), diff.mean())
    assert np.all(got[hole][:, 3] == 255)
    net.close()
    syn.close()


def test_inpaint_frame_without_holes(un):
    """IPD 0: every pixel is reached, the hole-cell list is empty, every convolution
    launch finds no band to compute, and the frame comes back byte for byte."""
    import paper_2506_15183_gb300 as yoro
    from paper_2506_15183_gb300 import scene

    cfg = scene.small_config().replace(w=200, h=136, ipd=0.0)
    c, d, _ = scene.render(cfg, 4)
    syn = yoro.Synthesizer(**cfg.camera())
    rgba = torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8, device="cuda")
    mask = torch.empty((cfg.h, cfg.w), dtype=torch.uint8, device="cuda")
    zt = torch.empty((cfg.h, cfg.w), dtype=torch.float32, device="cuda")
    dg = torch.from_numpy(d).cuda()
    yoro.yoro_synthesize_zt(syn.handle, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
    torch.cuda.synchronize()
    assert int(mask.sum()) == 0
    before = rgba.clone()
    net = _net(un, _weights(13), max_w=cfg.w, max_h=cfg.h)
    net.inpaint(rgba, mask, zt, dg, cfg.near)
    assert un.status() == 0
    assert torch.equal(rgba, before)
    net.close()
    syn.close()


def test_inpaint_reused_network_matches_a_fresh_one(un):
    """A network that just repainted another frame (a different scene, more hole cells)
    repaints the next one to the same bytes as a network that never ran: nothing of the
    earlier call's tiles or barrier phases carries over."""
    import paper_2506_15183_gb300 as yoro

    p = _weights(17)
    results = []
    for first in (None, 7):
        net = _net(un, p, max_w=256, max_h=256)
        if first is not None:
            cfg0, c0, d0, _ = _frame_tiles(first)
            syn0 = yoro.Synthesizer(**cfg0.camera())
            r0 = torch.empty((256, 256, 4), dtype=torch.uint8, device="cuda")
            m0 = torch.empty((256, 256), dtype=torch.uint8, device="cuda")
            z0 = torch.empty((256, 256), dtype=torch.float32, device="cuda")
            d0g = torch.from_numpy(d0).cuda()
            yoro.yoro_synthesize_zt(syn0.handle, torch.from_numpy(c0).cuda(), d0g, r0, m0, z0)
            net.inpaint(r0, m0, z0, d0g, cfg0.near)
            syn0.close()
        cfg, c, d, _ = _frame_tiles(2)
        syn = yoro.Synthesizer(**cfg.camera())
        rgba = torch.empty((256, 256, 4), dtype=torch.uint8, device="cuda")
        mask = torch.empty((256, 256), dtype=torch.uint8, device="cuda")
        zt = torch.empty((256, 256), dtype=torch.float32, device="cuda")
        dg = torch.from_numpy(d).cuda()
        yoro.yoro_synthesize_zt(syn.handle, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
        net.inpaint(rgba, mask, zt, dg, cfg.near)
        assert un.status() == 0
        results.append(rgba.cpu().numpy())
        net.close()
        syn.close()
    assert np.array_equal(results[0], results[1])


def test_inpaint_batch_matches_single_frames(un):
    """yoro_unet_inpaint_batch: frames of three sizes and scenes in one call (and, with a
    network whose buffers hold fewer cells than the batch, in several passes) give each
    frame the bytes yoro_unet_inpaint gives it alone."""
    import paper_2506_15183_gb300 as yoro

    p = _weights(19)
    specs = [(5, 256, 256), (6, 200, 136), (7, 256, 192)]
    inputs = []
    for seed, w, h in specs:
        cfg, c, d, _ = _frame_tiles(seed, w, h)
        syn = yoro.Synthesizer(**cfg.camera())
        rgba = torch.empty((h, w, 4), dtype=torch.uint8, device="cuda")
        mask = torch.empty((h, w), dtype=torch.uint8, device="cuda")
        zt = torch.empty((h, w), dtype=torch.float32, device="cuda")
        dg = torch.from_numpy(d).cuda()
        yoro.yoro_synthesize_zt(syn.handle, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
        syn.close()
        inputs.append((rgba, mask, zt, dg, cfg.near))
    torch.cuda.synchronize()
    single = []
    net = _net(un, p, max_w=256, max_h=256)
    for rgba, mask, zt, dg, near in inputs:
        r = rgba.clone()
        net.inpaint(r, mask, zt, dg, near)
        single.append(r)
    for max_tiles in (0, 20):  # 0: one pass (capacity 16 cells x 3 frames fits 48); 20: several
        net2 = _net(un, p, max_tiles=max_tiles or 48, max_w=256, max_h=256)
        outs = [(rgba.clone(), mask, zt, dg, near) for rgba, mask, zt, dg, near in inputs]
        net2.inpaint_batch(outs)
        assert un.status() == 0
        for (r, *_), ref_r in zip(outs, single):
            assert torch.equal(r, ref_r)
        net2.close()
    net.close()


def test_inpaint_batch_rejects_before_running(un):
    """A frame larger than the network takes makes the whole call fail with
    YORO_ETOOBIG, and no frame of it is touched."""
    import paper_2506_15183_gb300 as yoro

    cfg, c, d, _ = _frame_tiles(5, 256, 256)
    syn = yoro.Synthesizer(**cfg.camera())
    rgba = torch.empty((256, 256, 4), dtype=torch.uint8, device="cuda")
    mask = torch.empty((256, 256), dtype=torch.uint8, device="cuda")
    zt = torch.empty((256, 256), dtype=torch.float32, device="cuda")
    dg = torch.from_numpy(d).cuda()
    yoro.yoro_synthesize_zt(syn.handle, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
    torch.cuda.synchronize()
    before = rgba.clone()
    net = _net(un, _weights(3), max_w=128, max_h=128)
    small = torch.zeros((64, 64, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(yoro.YoroError):
        net.inpaint_batch([(small, torch.ones((64, 64), dtype=torch.uint8, device="cuda"),
                            torch.zeros((64, 64), device="cuda"), torch.ones((64, 64), device="cuda"), 0.05),
                           (rgba, mask, zt, dg, cfg.near)])
    torch.cuda.synchronize()
    assert torch.equal(rgba, before) and int(small.sum()) == 0
    net.close()
    syn.close()
