"""The debug-bounds build on the GPU: parity with every access range-checked, and the
status word's reporting path (needs a GPU).

The check runs in a child process because a process loads one build of the library;
the parent keeps the release build for the other GPU tests."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_bounds_build_parity_and_status_word():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_check.py")], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug-bounds OK" in r.stdout
