"""The C ABI library: builds, loads without a GPU, exports every declared entry point,
and rejects bad arguments before touching the device (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(HEADER_DIR, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(yoro_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_15183_gb300 import _build
    import paper_2506_15183_gb300 as yoro

    _build.build_cuda()
    return yoro.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("yoro_create", "yoro_destroy", "yoro_synthesize", "yoro_synthesize_batch",
                     "yoro_stream_status", "yoro_last_create_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2506_15183_gb300 import _build

    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(yoro_\w+)\b", out))
    for name in _declared():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_debug_bounds_build_exports_the_same_boundary(lib):
    """The debug-bounds variant builds from the same sources, exports every declared
    entry point and says which build it is; the release library says it is not."""
    from paper_2506_15183_gb300 import _build

    path = _build.build_cuda(debug=True)
    assert path == _build.DEBUG_LIB and path != _build.LIB
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(yoro_\w+)\b", out))
    assert set(_declared()) <= exported
    assert lib.yoro_debug_bounds_enabled() == 0
    probe = "import ctypes, sys; print(ctypes.CDLL(sys.argv[1]).yoro_debug_bounds_enabled())"
    r = subprocess.run([sys.executable, "-c", probe, path], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "1", r.stderr


def test_library_is_built_for_sm_103a(lib):
    from paper_2506_15183_gb300 import _build

    assert "arch=compute_103a,code=sm_103a" in _build.ARCH
    _build.build_cuda(force=True)
    log = open(os.path.join(_build.BUILD, "ptxas.log")).read()
    assert "for 'sm_103a'" in log and "fused_single" in log


def test_create_rejects_bad_camera_without_touching_the_device(lib):
    import paper_2506_15183_gb300 as yoro

    bad = [(-1, 4, 1, 1, 0, 0, 0.06, 0.05, 1000), (4, 4, 0, 1, 0, 0, 0.06, 0.05, 1000),
           (4, 4, 1, 1, 0, 0, -0.1, 0.05, 1000), (4, 4, 1, 1, 0, 0, 0.06, 0.0, 1000),
           (4, 4, 1, 1, 0, 0, 0.06, 2.0, 1.0), (4, 4, float("nan"), 1, 0, 0, 0.06, 0.05, 1000),
           (65536, 65536, 1, 1, 0, 0, 0.06, 0.05, 1000)]
    for args in bad:
        assert lib.yoro_create(*args) is None
        assert lib.yoro_last_create_error() == 1
        with pytest.raises(yoro.YoroError):
            yoro.yoro_create(*args)


def test_create_ex_rejects_bad_options_without_touching_the_device(lib):
    import paper_2506_15183_gb300 as yoro

    for kr, nf in ((2, 0), (0, 0), (17, 0), (-1, 0), (3, 2)):
        opt = yoro._Options(kr, nf)
        assert lib.yoro_create_ex(64, 64, 32.0, 32.0, 32.0, 32.0, 0.06, 0.05, 1000.0, opt) is None
        assert lib.yoro_last_create_error() == 1


def test_create_imb_rejects_bad_buffer_arguments_without_touching_the_device(lib):
    import paper_2506_15183_gb300 as yoro

    opt = yoro._Options(3, 0)
    for div, interp in ((0, 0), (3, 0), (32, 0), (-2, 0), (2, 2), (4, -1)):
        assert lib.yoro_create_imb(64, 64, 32.0, 32.0, 32.0, 32.0, 0.06, 0.05, 1000.0, opt, div, interp) is None
        assert lib.yoro_last_create_error() == 1


def test_create_pose_rejects_bad_arguments_without_touching_the_device(lib):
    import ctypes

    import paper_2506_15183_gb300 as yoro

    opt = yoro._Options(3, 0)
    eye = (ctypes.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    pos = (ctypes.c_float * 3)(0.063, 0, 0)
    bad_rot = (ctypes.c_float * 9)(1, 0, 0, 0, float("nan"), 0, 0, 0, 1)
    bad_pos = (ctypes.c_float * 3)(0.063, float("inf"), 0)
    for args in ((eye, None), (None, pos), (bad_rot, pos), (eye, bad_pos)):
        assert lib.yoro_create_pose(64, 64, 32.0, 32.0, 32.0, 32.0, args[0], args[1], 0.05, 1000.0, opt) is None
        assert lib.yoro_last_create_error() == 1
    assert lib.yoro_create_pose(64, 64, 32.0, 0.0, 32.0, 32.0, eye, pos, 0.05, 1000.0, opt) is None


def test_server_rejects_bad_arguments_without_touching_the_device(lib):
    from paper_2506_15183_gb300 import server

    sl = server._lib()
    assert sl.yoro_server_create(0, 8) is None and sl.yoro_last_create_error() == 1
    assert sl.yoro_server_create(1 << 30, 0) is None and sl.yoro_last_create_error() == 1
    assert sl.yoro_server_create(1 << 30, 5000) is None and sl.yoro_last_create_error() == 1
    assert sl.yoro_server_admit(None, 64, 64, 32.0, 32.0, 32.0, 32.0, 0.06, 0.05, 1000.0, 2) == -1
    assert sl.yoro_server_leave(None, 0) == 1
    assert sl.yoro_server_submit(None, 0, 0, 0) == 1
    assert sl.yoro_server_poll(None, None, 4) == 0
    assert sl.yoro_server_drain(None, 10) == 1
    assert sl.yoro_server_memory_used(None) == 0
    sl.yoro_server_destroy(None)


def test_null_handle_and_strings(lib):
    assert lib.yoro_synthesize(None, None, None, None, None, None) == 1
    assert lib.yoro_synthesize_unfused(None, None, None, None, None, None) == 1
    assert lib.yoro_synthesize_host(None, None, None, None, None, None) == 1
    assert lib.yoro_synthesize_batch(-1, None, None) == 1
    assert lib.yoro_tune_batch(0, None, 1, None, None) == 1
    assert lib.yoro_tune_batch(-3, None, 1, None, None) == 1
    assert lib.yoro_batch_band(0) == 0
    lib.yoro_reset_tuning()
    lib.yoro_destroy(None)
    for code in range(7):
        assert lib.yoro_status_string(code)


def test_inpainter_entry_points_check_arguments_without_a_gpu(lib):
    """The inpainter's parameter count matches the package's layer table, and bad
    arguments are refused before anything touches the device."""
    from paper_2506_15183_gb300 import unet, weights

    assert unet.param_count() == weights.count()
    L = unet._lib_net()
    assert not L.yoro_unet_create(None, weights.count(), 1, 64, 64)
    # null pointers and unsupported shapes (Cout 48, Cin 16) of the layer call
    assert L.yoro_unet_conv3x3(None, 1, 64, 64, 32, None, None, None, 32, 32, 0, 0, 1, None) == 1
    assert L.yoro_unet_forward(None, None, 1, None, None) == 1
    assert L.yoro_unet_inpaint(None, 64, 64, 0.05, None, None, None, None, None) == 1
