"""The batched workload: 64 frames of four per-eye sizes in one launch (needs a GPU).

16 frames each of 1024x1024, 1440x1600, 1832x1920 and 2064x2208, each an independent
seeded scene (50-300 primitives, IPD uniform in 0.055-0.072 m), synthesized by one
yoro_synthesize_batch call; every frame must equal the CPU oracle byte for byte.  The
same batch is also captured in a CUDA graph and replayed.
"""
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _render_and_ref(args):
    cfg, seed = args
    import oracle
    from paper_2506_15183_gb300 import scene

    c, d, _ = scene.render(cfg, seed, nthreads=2)
    ref = oracle.synthesize(c, d, cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.ipd, cfg.near, cfg.far)
    return c, d, ref


@pytest.fixture(scope="module")
def batch64():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import multiprocessing as mp

    import oracle
    import paper_2506_15183_gb300 as yoro
    from paper_2506_15183_gb300 import _build, scene

    _build.build_cuda()
    oracle.build()
    scene.build()
    yoro.load_library()
    specs = scene.batch_configs(64)
    workers = max(1, min(16, (os.cpu_count() or 2)))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        data = list(ex.map(_render_and_ref, specs))
    frames = []
    for (cfg, seed), (c, d, ref) in zip(specs, data):
        frames.append(dict(cfg.camera(), color=torch.from_numpy(c).cuda(), depth=torch.from_numpy(d).cuda(),
                           out_color=torch.empty((cfg.h, cfg.w, 4), dtype=torch.uint8, device="cuda"),
                           out_mask=torch.empty((cfg.h, cfg.w), dtype=torch.uint8, device="cuda"), ref=ref))
    return yoro, frames


def _check(frames):
    for i, fr in enumerate(frames):
        ro, rm = fr["ref"]
        assert np.array_equal(fr["out_color"].cpu().numpy(), ro), f"frame {i} color"
        assert np.array_equal(fr["out_mask"].cpu().numpy(), rm), f"frame {i} mask"


def test_batch_of_64_mixed_frames_bit_exact(batch64):
    yoro, frames = batch64
    sizes = {(fr["w"], fr["h"]) for fr in frames}
    assert sizes == {(1024, 1024), (1440, 1600), (1832, 1920), (2064, 2208)}
    for fr in frames:
        fr["out_color"].fill_(3)
        fr["out_mask"].fill_(3)
    yoro.yoro_synthesize_batch(frames)
    torch.cuda.synchronize()
    assert yoro.yoro_stream_status(None) == 0
    _check(frames)


def test_batch_replays_from_a_cuda_graph(batch64):
    yoro, frames = batch64
    sub = frames[:8]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        yoro.yoro_synthesize_batch(sub, stream=s)  # warm-up outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        yoro.yoro_synthesize_batch(sub, stream=s)
    for fr in sub:
        fr["out_color"].fill_(9)
        fr["out_mask"].fill_(9)
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    _check(sub)


def test_tuned_band_is_used_and_stays_exact(batch64):
    """The autotuner picks one of its candidate band heights for the widest frame, later
    batch launches use it, results stay bit-exact, and a reset restores the default."""
    yoro, frames = batch64
    wmax = max(fr["w"] for fr in frames)
    yoro.yoro_reset_tuning()
    default = yoro.yoro_batch_band(wmax)
    assert default >= 1
    for fr in frames:
        fr["out_color"].zero_()
        fr["out_mask"].fill_(7)
    band = yoro.yoro_tune_batch(frames, reps=2)
    assert 1 <= band <= default
    assert yoro.yoro_batch_band(wmax) == band
    torch.cuda.synchronize()
    _check(frames)  # the tuner's own launches already wrote the result
    for fr in frames:
        fr["out_color"].zero_()
    yoro.yoro_synthesize_batch(frames)
    torch.cuda.synchronize()
    _check(frames)
    yoro.yoro_reset_tuning()
    assert yoro.yoro_batch_band(wmax) == default
