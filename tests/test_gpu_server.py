"""The serving loop (include/yoro_server.h) on the GPU: continuous batching of several
streams gives every frame the same bytes as the frame alone and as the CPU oracle;
admission respects the memory budget (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_15183_gb300 import scene

pytestmark = pytest.mark.gpu

SIZES = [(1440, 1600), (1832, 1920), (2064, 2208), (1832, 1920), (1440, 1600), (2064, 2208), (1024, 1024),
         (1832, 1920)]


@pytest.fixture(scope="module")
def srv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_15183_gb300 as y
    from paper_2506_15183_gb300 import _build
    from paper_2506_15183_gb300 import server

    _build.build_cuda()
    y.load_library()
    return server


def _cfg(i):
    w, h = SIZES[i]
    return scene.quest_config().replace(w=w, h=h, n_prims=100 + 10 * i, ipd=0.058 + 0.002 * i)


def _frame(i, pose):
    cfg = _cfg(i)
    c, d, _ = scene.render(cfg, 300 + 17 * i + pose, eye_x=0.01 * pose)
    return cfg, c, d


def _bytes_per_slot(w, h):
    n = w * h
    a = lambda b: (b + 255) // 256 * 256  # noqa: E731
    return 3 * a(4 * n) + a(n)


def test_frames_alone_and_in_the_mix_are_identical(srv):
    cfg, c, d = _frame(1, 0)
    cam = cfg.camera()
    # alone
    s1 = srv.Server(1 << 30, max_batch=8)
    a = s1.admit(**cam, slots=1)
    ci, di, co, mo = s1.slot(a, 0)
    ci.copy_(torch.from_numpy(c))
    di.copy_(torch.from_numpy(d))
    torch.cuda.synchronize()
    s1.submit(a, 0, tag=7)
    s1.drain()
    done = s1.poll()
    assert len(done) == 1 and done[0].tag == 7 and done[0].status == 0 and done[0].batch_frames == 1
    alone = (co.cpu().numpy().copy(), mo.cpu().numpy().copy())
    ref = oracle.synthesize(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"], cam["near"], cam["far"])
    assert np.array_equal(alone[0], ref[0]) and np.array_equal(alone[1], ref[1])
    s1.close()
    # in a mix of eight streams, three rounds, the same frame in round 1 of stream 1
    s2 = srv.Server(8 << 30, max_batch=16)
    ids, frames = [], {}
    for i in range(len(SIZES)):
        ids.append(s2.admit(**_cfg(i).camera(), slots=3))
    for rnd in range(3):
        for i, sid in enumerate(ids):
            fcfg, fc, fd = (cfg, c, d) if (i == 1 and rnd == 1) else _frame(i, rnd + 1)
            ci, di, _, _ = s2.slot(sid, rnd)
            ci.copy_(torch.from_numpy(fc))
            di.copy_(torch.from_numpy(fd))
            frames[(sid, rnd)] = (fcfg, fc, fd)
        torch.cuda.synchronize()
        for i, sid in enumerate(ids):
            s2.submit(sid, rnd, tag=rnd * 100 + i)
    s2.drain()
    done = s2.poll(4096)
    assert sorted(r.tag for r in done) == sorted(rnd * 100 + i for rnd in range(3) for i in range(len(ids)))
    assert all(r.status == 0 and r.submit_ns <= r.launch_ns <= r.done_ns for r in done)
    assert max(r.batch_frames for r in done) > 1  # frames of several streams shared launches
    _, _, co, mo = s2.slot(ids[1], 1)
    assert np.array_equal(co.cpu().numpy(), alone[0]) and np.array_equal(mo.cpu().numpy(), alone[1])
    for (sid, rnd), (fcfg, fc, fd) in frames.items():  # every frame of the mix against the oracle
        fc_ = fcfg.camera()
        r = oracle.synthesize(fc, fd, fc_["fx"], fc_["fy"], fc_["cx"], fc_["cy"], fc_["ipd"], fc_["near"], fc_["far"])
        _, _, co, mo = s2.slot(sid, rnd)
        assert np.array_equal(co.cpu().numpy(), r[0]) and np.array_equal(mo.cpu().numpy(), r[1]), (sid, rnd)
    s2.close()


def test_admission_follows_the_memory_budget(srv):
    import paper_2506_15183_gb300 as y

    cam = _cfg(1).camera()
    per = _bytes_per_slot(cam["w"], cam["h"]) * 2
    s = srv.Server(2 * per + per // 2, max_batch=4)
    a = s.admit(**cam, slots=2)
    b = s.admit(**cam, slots=2)
    assert s.memory_used() == 2 * per
    with pytest.raises(y.YoroError) as e:
        s.admit(**cam, slots=2)
    assert e.value.code == 3  # YORO_ENOMEM
    s.leave(a)
    assert s.memory_used() == per
    c = s.admit(**cam, slots=2)
    assert c not in (a, b)
    with pytest.raises(y.YoroError):
        s.submit(a, 0)  # a stream that left
    with pytest.raises(y.YoroError):
        s.submit(c, 5)  # no such slot
    s.close()


def test_leaving_with_frames_in_flight_completes_them_first(srv):
    """A stream that leaves while its frames are queued or running: leave() waits for
    them, frees its slots, and their completions stay available to poll()."""
    cfg, c, d = _frame(6, 0)
    cam = cfg.camera()
    s = srv.Server(1 << 30, max_batch=4)
    a = s.admit(**cam, slots=3)
    ref = oracle.synthesize(c, d, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"], cam["near"], cam["far"])
    for k in range(3):
        ci, di, _, _ = s.slot(a, k)
        ci.copy_(torch.from_numpy(c))
        di.copy_(torch.from_numpy(d))
    torch.cuda.synchronize()
    for k in range(3):
        s.submit(a, k, tag=40 + k)
    s.leave(a)  # no drain first
    assert s.memory_used() == 0
    done = s.poll()
    assert sorted(r.tag for r in done) == [40, 41, 42] and all(r.status == 0 for r in done)
    # the server keeps serving: a new stream gets the oracle's bytes
    b = s.admit(**cam, slots=1)
    ci, di, co, mo = s.slot(b, 0)
    ci.copy_(torch.from_numpy(c))
    di.copy_(torch.from_numpy(d))
    torch.cuda.synchronize()
    s.submit(b, 0, tag=50)
    s.drain()
    assert [r.tag for r in s.poll()] == [50]
    assert np.array_equal(co.cpu().numpy(), ref[0]) and np.array_equal(mo.cpu().numpy(), ref[1])
    s.close()


# ---- learned inpainting in the serving loop, and host-side faults --------------------

def _fill_slot(s, sid, k, c, d):
    ci, di, _, _ = s.slot(sid, k)
    ci.copy_(torch.from_numpy(c))
    di.copy_(torch.from_numpy(d))


def _small(i):
    cfg = scene.small_config().replace(w=256 + 64 * (i % 2), h=256, ipd=0.06 + 0.002 * i)
    c, d, _ = scene.render(cfg, 700 + i)
    return cfg, c, d


def test_learned_stream_in_the_mix_equals_the_frame_alone(srv):
    """A stream with learned inpainting shares batches with plain streams: its frame gets
    the bytes of yoro_synthesize_zt + yoro_unet_inpaint on the frame alone, the plain
    frames the oracle's, and each completion says which fill it got."""
    import paper_2506_15183_gb300 as y
    from paper_2506_15183_gb300 import unet as un
    from paper_2506_15183_gb300 import weights as W

    net = un.Inpainter(W.init_params(4), max_w=320, max_h=256)
    frames = [_small(i) for i in range(3)]
    # alone
    cfg, c, d = frames[1]
    hdl = y.yoro_create(**cfg.camera())
    rgba = torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8, device="cuda")
    mask = torch.empty((cfg.h, cfg.w), dtype=torch.uint8, device="cuda")
    zt = torch.empty((cfg.h, cfg.w), dtype=torch.float32, device="cuda")
    dg = torch.from_numpy(d).cuda()
    y.yoro_synthesize_zt(hdl, torch.from_numpy(c).cuda(), dg, rgba, mask, zt)
    net.inpaint(rgba, mask, zt, dg, cfg.near)
    torch.cuda.synchronize()
    alone = rgba.cpu().numpy()
    y.yoro_destroy(hdl)
    # in the mix
    s = srv.Server(1 << 30, max_batch=8)
    s.set_inpainter(net)
    ids = [s.admit(**f[0].camera(), slots=2, learned=(i == 1)) for i, f in enumerate(frames)]
    for sid, (fcfg, fc, fd) in zip(ids, frames):
        _fill_slot(s, sid, 0, fc, fd)
    torch.cuda.synchronize()
    for k, sid in enumerate(ids):
        s.submit(sid, 0, tag=k)
    s.drain()
    done = {r.tag: r for r in s.poll()}
    assert all(done[k].status == 0 for k in range(3))
    assert [done[k].inpainted for k in range(3)] == [0, 1, 0]
    assert np.array_equal(s.slot(ids[1], 0)[2].cpu().numpy(), alone)
    assert not np.array_equal(alone, oracle.synthesize(c, d, cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.ipd, cfg.near,
                                                       cfg.far)[0])  # the network did repaint
    for i in (0, 2):
        fcfg, fc, fd = frames[i]
        ref = oracle.synthesize(fc, fd, fcfg.fx, fcfg.fy, fcfg.cx, fcfg.cy, fcfg.ipd, fcfg.near, fcfg.far)
        assert np.array_equal(s.slot(ids[i], 0)[2].cpu().numpy(), ref[0])
    s.close()
    net.close()


def test_learned_stream_without_an_inpainter_keeps_the_papers_fill(srv):
    cfg, c, d = _small(0)
    s = srv.Server(1 << 30, max_batch=4)
    a = s.admit(**cfg.camera(), slots=1, learned=True)
    _fill_slot(s, a, 0, c, d)
    torch.cuda.synchronize()
    s.submit(a, 0, tag=1)
    s.drain()
    (r,) = s.poll()
    assert r.status == 0 and r.inpainted == 0
    ref = oracle.synthesize(c, d, cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.ipd, cfg.near, cfg.far)
    assert np.array_equal(s.slot(a, 0)[2].cpu().numpy(), ref[0])
    s.close()


def test_drain_times_out_while_nothing_can_run(srv):
    """The scheduler is paused, so a submitted frame cannot complete: drain() gives up
    after its time limit with YORO_ETIMEOUT; resumed, the frame completes normally."""
    import paper_2506_15183_gb300 as y

    cfg, c, d = _small(1)
    s = srv.Server(1 << 30, max_batch=4)
    a = s.admit(**cfg.camera(), slots=1)
    _fill_slot(s, a, 0, c, d)
    torch.cuda.synchronize()
    s.pause(True)
    s.submit(a, 0, tag=9)
    with pytest.raises(y.YoroError) as e:
        s.drain(50)
    assert e.value.code == 7  # YORO_ETIMEOUT
    assert s.poll() == []
    s.pause(False)
    s.drain()
    (r,) = s.poll()
    assert r.tag == 9 and r.status == 0
    s.close()


def test_cancel_drops_queued_frames_and_frees_their_slots(srv):
    import paper_2506_15183_gb300 as y

    cfg, c, d = _small(2)
    s = srv.Server(1 << 30, max_batch=4)
    a = s.admit(**cfg.camera(), slots=3)
    b = s.admit(**cfg.camera(), slots=1)
    for k in range(3):
        _fill_slot(s, a, k, c, d)
    _fill_slot(s, b, 0, c, d)
    torch.cuda.synchronize()
    s.pause(True)
    for k in range(3):
        s.submit(a, k, tag=k)
    s.submit(b, 0, tag=10)
    assert s.cancel(a) == 3
    done = s.poll()
    assert sorted(r.tag for r in done) == [0, 1, 2]
    assert all(r.status == 8 and r.batch_frames == 0 for r in done)  # YORO_ECANCELED
    s.submit(a, 1, tag=11)  # the slot is free again
    s.pause(False)
    s.drain()
    assert sorted(r.tag for r in s.poll()) == [10, 11]
    with pytest.raises(y.YoroError):
        s.cancel(99)
    s.close()


def test_an_oversized_frame_is_refused_at_admission(srv):
    import paper_2506_15183_gb300 as y

    s = srv.Server(1 << 34, max_batch=4)
    w = y.yoro_max_fused_width() + 32
    with pytest.raises(y.YoroError) as e:
        s.admit(w=w, h=64, fx=w / 2, fy=w / 2, cx=w / 2, cy=32, ipd=0.063, slots=1)
    assert e.value.code == 6  # YORO_ETOOBIG
    assert s.memory_used() == 0
    s.close()


def test_the_feeder_submits_from_device_sources(srv):
    """yoro_server_feed: the server's own thread copies source frames into free slots and
    submits them, unpaced and paced; every frame gets the oracle's bytes for its source."""
    frames = [_small(3), _small(5)]
    cfg = frames[0][0]
    s = srv.Server(1 << 30, max_batch=8)
    a = s.admit(**cfg.camera(), slots=2)
    src = [(torch.from_numpy(c).cuda(), torch.from_numpy(d).cuda()) for _, c, d in frames]
    torch.cuda.synchronize()
    s.feed(a, src, nframes=6, tag0=100)
    s.drain()
    got = []
    while len(got) < 6:
        got += s.poll()
        s.drain()
    assert sorted(r.tag for r in got) == list(range(100, 106)) and all(r.status == 0 for r in got)
    # the last frame sent (tag 105) was source 1; its slot holds that frame's result
    last = max(got, key=lambda r: r.tag)
    _, fc, fd = frames[1]  # synthesized with the stream's camera
    ref = oracle.synthesize(fc, fd, cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.ipd, cfg.near, cfg.far)
    assert np.array_equal(s.slot(a, last.slot)[2].cpu().numpy(), ref[0])
    # paced at 200 Hz: submissions at least ~5 ms apart
    s.feed(a, src, nframes=5, hz=200.0, tag0=200)
    import time

    t0 = time.time()
    paced = []
    while len(paced) < 5 and time.time() - t0 < 10:
        paced += s.poll()
        time.sleep(0.002)
    assert sorted(r.tag for r in paced) == list(range(200, 205))
    sub = sorted(r.submit_ns for r in paced)
    assert min(b - a_ for a_, b in zip(sub, sub[1:])) >= 4_000_000
    s.feed_stop()
    s.close()
