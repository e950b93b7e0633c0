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
    for sid, rnd in [(ids[0], 0), (ids[2], 2), (ids[6], 1)]:  # a few others against the oracle
        fcfg, fc, fd = frames[(sid, rnd)]
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
