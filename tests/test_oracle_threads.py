"""The all-core build of the oracle (the same C source compiled with -fopenmp, rows
split over the host's cores) gives byte for byte what the one-thread build gives.  It
is the CPU baseline's all-core leg; its arithmetic is the oracle's own."""
import numpy as np

import oracle
from paper_2506_15183_gb300 import scene


def _both(cfg, seed, **kw):
    c, d, _ = scene.render(cfg, seed)
    args = (c, d, cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.ipd, cfg.near, cfg.far)
    return oracle.synthesize(*args, **kw), oracle.synthesize(*args, all_cores=True, **kw)


def test_all_core_build_uses_threads_and_the_single_build_does_not():
    assert oracle.threads(all_cores=False) == 1
    assert oracle.threads(all_cores=True) >= 1


def test_all_core_build_is_byte_identical_small():
    for seed in (1, 2, 3):
        (o1, m1), (o2, m2) = _both(scene.small_config(), seed)
        assert np.array_equal(o1, o2) and np.array_equal(m1, m2)
        assert m1.any()


def test_all_core_build_is_byte_identical_variant_kernel():
    (o1, m1), (o2, m2) = _both(scene.small_config(), 4, kernel_rows=5, nearest_first=True)
    assert np.array_equal(o1, o2) and np.array_equal(m1, m2)


def test_all_core_build_is_byte_identical_quest_frame():
    (o1, m1), (o2, m2) = _both(scene.quest_config(), 2)
    assert np.array_equal(o1, o2) and np.array_equal(m1, m2)
