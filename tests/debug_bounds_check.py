"""Parity run of the debug-bounds build (``libyoro_debug.so``) in a process of its own.

Run by ``test_gpu_debug_bounds.py`` as ``python tests/debug_bounds_check.py``: the
process loads the debug-bounds library before any other call, synthesizes frames that
exercise every kernel (fused single-frame launch with the default and variant kernels
and with the warped-depth output, the batch launch with and without it, the unfused
launch, the intermediate-buffer and general-pose launches; tall bands,
ragged widths, a wide-disparity camera), and checks for each that the status word stayed clear (no range check failed)
and that the result still equals the CPU oracle byte for byte.  Then the self-test
kernel must raise ``YORO_EDEVICE`` exactly once.  Prints ``debug-bounds OK`` at the end.
"""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import paper_2506_15183_gb300 as yoro  # noqa: E402
from paper_2506_15183_gb300 import _build, scene  # noqa: E402

DEV = "cuda:0"
EDEVICE = 5


def _ref(c, d, cam, kernel_rows=3, nearest_first=False):
    return oracle.synthesize(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"], cam["near"], cam["far"],
                             kernel_rows=kernel_rows, nearest_first=nearest_first)


def _same(got, ref, what):
    bad = np.nonzero((got[0] != ref[0]).any(axis=-1) | (got[1] != ref[1]))
    assert bad[0].size == 0, f"{what}: {bad[0].size} pixels differ, first at {bad[0][0]},{bad[1][0]}"


def _single(c, d, cam, kernel_rows=3, nearest_first=False, what=""):
    ref = _ref(c, d, cam, kernel_rows, nearest_first)
    for unfused in (False, True):
        syn = yoro.Synthesizer(**cam, kernel_rows=kernel_rows, nearest_first=nearest_first)
        out, mask = syn(torch.from_numpy(c).to(DEV), torch.from_numpy(d).to(DEV), unfused=unfused)
        st = syn.status()
        assert st == 0, f"{what} unfused={unfused}: status {yoro.STATUS.get(st, st)}"
        _same((out.cpu().numpy(), mask.cpu().numpy()), ref, f"{what} unfused={unfused}")
        syn.close()


def _ragged(h, w, seed, ipd=0.063, fx=None):
    rng = np.random.default_rng(seed)
    runs = rng.uniform(0.05, 6.0, (h, (w + 6) // 7)).astype(np.float32)
    d = np.ascontiguousarray(np.repeat(runs, 7, axis=1)[:, :w])
    c = rng.integers(0, 256, (h, w, 4), dtype=np.uint8)
    fx = w / 2.0 if fx is None else fx
    cam = dict(w=w, h=h, fx=fx, fy=fx, cx=w / 2.0, cy=h / 2.0, ipd=ipd, near=0.05, far=1000.0)
    return c, d, cam


def main() -> None:
    if not torch.cuda.is_available():
        raise SystemExit("no CUDA device")
    _build.build_cuda(debug=True)
    scene.build()
    lib = yoro.load_library(debug=True)
    assert lib.yoro_debug_bounds_enabled() == 1
    assert yoro.yoro_stream_status(None) == 0  # nothing recorded yet

    cfg = scene.quest_config()
    c, d, _ = scene.render(cfg, 4)
    _single(c, d, cfg.camera(), what="quest frame")
    _single(c, d, cfg.camera(), 5, True, what="quest frame h=5 nearest-first")

    small = scene.small_config()
    for seed in (1, 2):
        c, d, _ = scene.render(small, seed)
        for kr, nf in ((3, False), (1, True), (9, False)):
            _single(c, d, small.camera(), kr, nf, what=f"small seed {seed} h={kr} nf={nf}")

    c, d, cam = _ragged(9000, 64, 5, ipd=0.1, fx=32.0)
    _single(c, d, cam, 7, True, what="tall narrow h=7")
    _single(c, d, cam, what="tall narrow")
    for h, w in ((4, 8), (16, 16), (37, 1), (37, 31), (37, 33), (37, 1000), (37, 2049)):
        c, d, cam = _ragged(h, w, w)
        _single(c, d, cam, what=f"{w}x{h}")
    c, d, cam = _ragged(64, 777, 9, ipd=2.0, fx=5000.0)  # targets far outside the frame
    _single(c, d, cam, what="wide disparity")

    # the row-downsampled intermediate buffer
    c, d, _ = scene.render(small, 3)
    cam = small.camera()
    for div, interp in ((4, True), (16, False)):
        ref = oracle.synthesize_imb(c, d, cam["fx"], cam["ipd"], cam["near"], cam["far"], div, interp)
        syn = yoro.Synthesizer(**cam, imbuffer_div=div, interpolate=interp)
        out, mask = syn(torch.from_numpy(c).to(DEV), torch.from_numpy(d).to(DEV))
        st = syn.status()
        assert st == 0, f"imbuffer {div} {interp}: status {yoro.STATUS.get(st, st)}"
        _same((out.cpu().numpy(), mask.cpu().numpy()), ref, f"imbuffer {div} {interp}")
        syn.close()
        # the same frame through the separate kernels
        syn = yoro.Synthesizer(**cam, imbuffer_div=div, interpolate=interp)
        out, mask = syn(torch.from_numpy(c).to(DEV), torch.from_numpy(d).to(DEV), unfused=True)
        st = syn.status()
        assert st == 0, f"imbuffer unfused {div} {interp}: status {yoro.STATUS.get(st, st)}"
        _same((out.cpu().numpy(), mask.cpu().numpy()), ref, f"imbuffer unfused {div} {interp}")
        syn.close()

    # a general second-eye pose (rotated, offset up)
    rot = np.array([[0.9998, 0.0, 0.02], [0.0, 1.0, 0.0], [-0.02, 0.0, 0.9998]], np.float32)
    pose = (rot, [0.063, 0.01, 0.0])
    ref = oracle.synthesize_pose(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], rot, pose[1], cam["near"],
                                 cam["far"])
    syn = yoro.Synthesizer(**cam, pose=pose)
    out, mask = syn(torch.from_numpy(c).to(DEV), torch.from_numpy(d).to(DEV))
    st = syn.status()
    assert st == 0, f"pose: status {yoro.STATUS.get(st, st)}"
    _same((out.cpu().numpy(), mask.cpu().numpy()), ref, "pose")
    syn.close()

    frames = []
    for i, (w, h) in enumerate(((1024, 1024), (1440, 1600), (333, 71), (1832, 1920))):
        c, d, cam = _ragged(h, w, 100 + i)
        frames.append(dict(cam, color=torch.from_numpy(c).to(DEV), depth=torch.from_numpy(d).to(DEV),
                           out_color=torch.empty((h, w, 4), dtype=torch.uint8, device=DEV),
                           out_mask=torch.empty((h, w), dtype=torch.uint8, device=DEV), ref=_ref(c, d, cam)))
    yoro.yoro_synthesize_batch(frames)
    st = yoro.yoro_stream_status(None)
    assert st == 0, f"batch: status {yoro.STATUS.get(st, st)}"
    for i, fr in enumerate(frames):
        _same((fr["out_color"].cpu().numpy(), fr["out_mask"].cpu().numpy()), fr["ref"], f"batch frame {i}")

    # the warped-depth instantiations: a single frame (yoro_synthesize_zt) and a batch
    # with a learned stream in the serving loop (the batch kernel writing warped depth)
    from paper_2506_15183_gb300 import server as srv

    for (h, w, seed) in ((64, 333, 7), (1920, 1832, 8)):
        c, d, cam = _ragged(h, w, seed)
        hdl = yoro.yoro_create(**cam)
        out = torch.empty((h, w, 4), dtype=torch.uint8, device=DEV)
        mask = torch.empty((h, w), dtype=torch.uint8, device=DEV)
        zt = torch.empty((h, w), dtype=torch.float32, device=DEV)
        yoro.yoro_synthesize_zt(hdl, torch.from_numpy(c).to(DEV), torch.from_numpy(d).to(DEV), out, mask, zt)
        st = yoro.yoro_stream_status(hdl)
        assert st == 0, f"synthesize_zt {w}x{h}: status {yoro.STATUS.get(st, st)}"
        _same((out.cpu().numpy(), mask.cpu().numpy()), _ref(c, d, cam), f"synthesize_zt {w}x{h}")
        yoro.yoro_destroy(hdl)
    c, d, cam = _ragged(71, 333, 11)
    s = srv.Server(1 << 28, max_batch=4)
    a = s.admit(**cam, slots=1, learned=True)
    b = s.admit(**cam, slots=1)
    for sid in (a, b):
        ci, di, _, _ = s.slot(sid, 0)
        ci.copy_(torch.from_numpy(c))
        di.copy_(torch.from_numpy(d))
    torch.cuda.synchronize()
    s.submit(a, 0, tag=1)
    s.submit(b, 0, tag=2)
    s.drain()
    assert all(r.status == 0 for r in s.poll())
    st = yoro.yoro_stream_status(None)
    assert st == 0, f"server batch with warped depth: status {yoro.STATUS.get(st, st)}"
    ref = _ref(c, d, cam)
    for sid in (a, b):
        _, _, co, mo = s.slot(sid, 0)
        _same((co.cpu().numpy(), mo.cpu().numpy()), ref, f"server stream {sid}")
    s.close()

    yoro.yoro_debug_selftest()
    assert yoro.yoro_stream_status(None) == EDEVICE, "the self-test code was not reported"
    assert yoro.yoro_stream_status(None) == 0, "the status word was not cleared by reading it"
    print("debug-bounds OK")


if __name__ == "__main__":
    main()
