"""yoro_synthesize_noalloc against yoro_synthesize, through the C ABI (needs a GPU).

The no-allocation entry point serves callers that must not call cudaMalloc where they
synthesize a frame (a compositor's per-frame callback, a plugin whose host owns the
device-memory budget); its z-buffer is an array inside the library that every call
shares.  Two calls in a row, a large frame then a smaller one, must each equal the
fused entry point's output and the CPU oracle's byte for byte: the second call must not
see what the first left in the shared array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_15183_gb300 import scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_15183_gb300 as yoro
    from paper_2506_15183_gb300 import _build

    _build.build_cuda()
    return yoro.load_library()


def _fused(cfg, c, d):
    import paper_2506_15183_gb300 as yoro

    syn = yoro.Synthesizer(**cfg.camera())
    out, mask = syn(c, d)
    torch.cuda.synchronize()
    syn.close()
    return out.cpu().numpy(), mask.cpu().numpy()


def test_noalloc_matches_fused_on_two_calls_in_a_row(lib):
    frames = []
    for cfg, seed in ((scene.quest_config(), 4), (scene.small_config(), 5)):
        c, d, _ = scene.render(cfg, seed)
        frames.append((cfg, torch.from_numpy(c).cuda(), torch.from_numpy(d).cuda()))
    stream = torch.cuda.current_stream().cuda_stream
    for cfg, c, d in frames:
        assert cfg.w * cfg.h <= lib.yoro_noalloc_max_pixels()
        out = torch.full((cfg.h, cfg.w, 4), 7, dtype=torch.uint8, device="cuda")
        mask = torch.full((cfg.h, cfg.w), 7, dtype=torch.uint8, device="cuda")
        cam = cfg.camera()
        rc = lib.yoro_synthesize_noalloc(cfg.w, cfg.h, cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["ipd"],
                                         cam["near"], cam["far"], c.data_ptr(), d.data_ptr(), out.data_ptr(),
                                         mask.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got_out, got_mask = out.cpu().numpy(), mask.cpu().numpy()
        ref_out, ref_mask = _fused(cfg, c, d)
        assert np.array_equal(got_out, ref_out)
        assert np.array_equal(got_mask, ref_mask)
        assert ref_mask.any()
        # and the definition itself
        or_out, or_mask = oracle.synthesize(c.cpu().numpy(), d.cpu().numpy(), cam["fx"], cam["fy"], cam["cx"],
                                            cam["cy"], cam["ipd"], cam["near"], cam["far"])
        assert np.array_equal(got_out, or_out)
        assert np.array_equal(got_mask, or_mask)


def test_noalloc_rejects_frames_beyond_its_array(lib):
    n = lib.yoro_noalloc_max_pixels()
    w = 4096
    h = n // w + 1
    dummy = torch.empty(16, dtype=torch.uint8, device="cuda")
    p = dummy.data_ptr()
    rc = lib.yoro_synthesize_noalloc(w, h, 2048.0, 2048.0, 2048.0, h / 2, 0.063, 0.05, 1000.0, p, p + 4096, p + 8192,
                                     p + 12288, None)
    assert rc == 6  # YORO_ETOOBIG, checked before any pointer is used
