"""Planted mistakes in the oracle must fail its pins (no GPU).

Each mutant is a copy of ``oracle/yoro_oracle.c`` with one plausible mistake (a
dropped term, a wrong sign, index or order), built into a temporary library and
loaded by a fresh pytest run of ``test_oracle_pins.py`` (or, for the intermediate
buffer's and the general reprojection's steps, ``test_oracle_imbuffer.py`` and
``test_oracle_pose.py``).  That run must fail: if it
passed, the pins would not tie the oracle to the paper at that point.
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "yoro_oracle.c")

MUTANTS = {
    "pixel_centre_dropped": ("float t = ((float)x + 0.5f) - disp;", "float t = (float)x - disp;"),
    "disparity_sign": ("float t = ((float)x + 0.5f) - disp;", "float t = ((float)x + 0.5f) + disp;"),
    "round_not_floor": ("float f = floorf(t);", "float f = rintf(t);"),
    "trunc_not_floor": ("float f = floorf(t);", "float f = truncf(t);"),
    "no_near_clamp": ("float c = fminf(fmaxf(z, near_), far_);\n            float disp = k / c;\n            float t = ((float)x",
                      "float c = fminf(z, far_);\n            float disp = k / c;\n            float t = ((float)x"),
    "farther_wins": ("if (src[o] < 0 || zc[i] < zt[o]) {", "if (src[o] < 0 || zc[i] > zt[o]) {"),
    "last_writer_wins_ties": ("if (src[o] < 0 || zc[i] < zt[o]) {", "if (src[o] < 0 || zc[i] <= zt[o]) {"),
    "t_from_occluder_edge": ("float t = (float)(R - u) / (float)wd;", "float t = (float)(u - L) / (float)wd;"),
    "weight_constant": ("float b = (0.3f * wrem) * t;", "float b = (0.25f * wrem) * t;"),
    "weight_half_term": ("float a = wrem * 0.5f;", "float a = wrem * 0.4f;"),
    "no_depth_gate": ("if (zt[q] < d_occ) continue;", ""),
    "gate_on_background_edge": ("float d_occ = (L >= 0) ? zt[(size_t)v * (size_t)w + (size_t)L] : 0.0f;",
                                "float d_occ = zt[(size_t)v * (size_t)w + (size_t)R];"),
    "column_order_swapped": ("int j = nearest_first ? R + s : jhi - s;", "int j = nearest_first ? jhi - s : R + s;"),
    "column_order_flag_ignored": ("int j = nearest_first ? R + s : jhi - s;", "int j = jhi - s;"),
    "kernel_one_column_short": ("int jhi = R + wd;", "int jhi = R + wd - 1;"),
    "single_row_kernel": ("for (int vv = v - hr; vv <= v + hr; ++vv) {", "for (int vv = v; vv <= v; ++vv) {"),
    "kernel_height_ignored": ("int hr = (kernel_rows - 1) / 2;", "int hr = 1;"),
    "divide_by_wrem": ("float den = 1.0f - wrem;", "float den = wrem;"),
    "fallback_to_occluder": ("    if (R < w)\n        memcpy(out, warped + 4 * ((size_t)v * (size_t)w + (size_t)R), 4);",
                             "    if (L >= 0)\n        memcpy(out, warped + 4 * ((size_t)v * (size_t)w + (size_t)L), 4);"),
    "alpha_not_filled": ("for (int c = 0; c < 4; ++c) {\n                float r", "for (int c = 0; c < 3; ++c) {\n                float r"),
    # the row-downsampled intermediate buffer, against its own pins
    "imb_cell_pixel_not_centre": ("int p = div * i + div / 2;", "int p = div * i;", "test_oracle_imbuffer.py"),
    "imb_target_cell_rounded": ("float tc = floorf(t / (float)div);", "float tc = rintf(t / (float)div);",
                                "test_oracle_imbuffer.py"),
    "imb_farther_cell_wins": ("if (wrow[j] < 0 || c < zrow[j]) {", "if (wrow[j] < 0 || c > zrow[j]) {",
                              "test_oracle_imbuffer.py"),
    "imb_place_in_cell_dropped": ("int sx = div * wrow[j] + (x - div * j);", "int sx = div * wrow[j];",
                                  "test_oracle_imbuffer.py"),
    "imb_neighbour_side_swapped": ("int nb = off < 0.0f ? j - 1 : j + 1;", "int nb = off < 0.0f ? j + 1 : j - 1;",
                                   "test_oracle_imbuffer.py"),
    "imb_shift_not_interpolated": ("D = drow[j] + (drow[nb] - drow[j]) * a;", "D = drow[j];",
                                   "test_oracle_imbuffer.py"),
    "imb_nearest_texel": ("float v = c0 + (c1 - c0) * f;", "float v = c0;", "test_oracle_imbuffer.py"),
    # the general reprojection, against its own pins
    "pose_rotation_transposed": ("float X = (rot[0] * q0 + rot[1] * q1) + rot[2] * q2;",
                                 "float X = (rot[0] * q0 + rot[3] * q1) + rot[6] * q2;", "test_oracle_pose.py"),
    "pose_farther_wins": ("if (win[o] < 0 || Z < zt[o]) {", "if (win[o] < 0 || Z > zt[o]) {", "test_oracle_pose.py"),
    "pose_row_centre_dropped": ("float py = (((float)y + 0.5f) - cy) * zc / fy;", "float py = ((float)y - cy) * zc / fy;",
                                "test_oracle_pose.py"),
    "pose_target_rounded": ("float u = floorf(fx * X / Z + cx);", "float u = rintf(fx * X / Z + cx);",
                            "test_oracle_pose.py"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name][:2]
    pins = MUTANTS[name][2] if len(MUTANTS[name]) > 2 else "test_oracle_pins.py"
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut_c = tmp_path / "mutant.c"
    mut_c.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-shared", "-fPIC", "-o", str(lib), str(mut_c), "-lm"])
    env = dict(os.environ, YORO_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"


UNET = os.path.join(ROOT, "oracle", "unet.py")
UNET_MUTANTS = {
    "unet_concat_order": ("a = np.concatenate([skips[l], upsample2(a)], axis=0)",
                          "a = np.concatenate([upsample2(a), skips[l]], axis=0)"),
    "unet_bf16_truncates": ("r = ((u + 0x7FFF + lsb) >> 16) << 16", "r = (u >> 16) << 16"),
    "unet_bf16_ties_up": ("r = ((u + 0x7FFF + lsb) >> 16) << 16", "r = ((u + 0x8000) >> 16) << 16"),
    "unet_no_bias": ("    return acc + b[:, None, None]\n\n\ndef conv1x1", "    return acc\n\n\ndef conv1x1"),
    "unet_padding_shifted": ("xp = np.zeros((c, h + 2, wd + 2), np.float32)\n    xp[:, 1:-1, 1:-1] = x",
                             "xp = np.zeros((c, h + 2, wd + 2), np.float32)\n    xp[:, :-2, 1:-1] = x"),
    "unet_activations_not_rounded": ("return bf16(np.maximum(x, np.float32(0.0)))",
                                     "return np.maximum(x, np.float32(0.0))"),
}


@pytest.mark.parametrize("name", sorted(UNET_MUTANTS))
def test_inpainter_pins_catch_mutant(name, tmp_path):
    """The same for the inpainter's definition (oracle/unet.py): a copy of the oracle
    package with one mistake comes first on the path of a fresh run of its pins."""
    import shutil

    old, new = UNET_MUTANTS[name]
    src = open(UNET).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    (tmp_path / "oracle" / "unet.py").write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=f"{tmp_path}{os.pathsep}{ROOT}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_unet.py")],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"


# Mistakes planted in the definition of the inpainter's training gradient
# (oracle/unet.py loss_and_grads); its finite-difference pin must catch each one.
GRAD_MUTANTS = {
    "grad_no_sigmoid_derivative": ("dzo = 2.0 * err / n * s_ * (1.0 - s_)", "dzo = 2.0 * err / n"),
    "grad_kernel_not_flipped": ('dxp[:, dy:dy + h, dx:dx + wd] += np.einsum("kc,khw->chw", w[:, :, dy, dx], dz)',
                                'dxp[:, dy:dy + h, dx:dx + wd] += np.einsum("kc,khw->chw", w[:, :, 2 - dy, 2 - dx], dz)'),
    "grad_skip_path_dropped": ("da = _maxpool_backward(src, da) + skip_grads.pop(l - 1)",
                               "da = _maxpool_backward(src, da) + 0 * skip_grads.pop(l - 1)"),
    "grad_pool_to_window_corner": ("first = np.argmax(win == win.max(axis=-1, keepdims=True), axis=-1)",
                                   "first = np.zeros(win.shape[:-1], int)"),
    "grad_upsample_averaged": ("da = d_up.reshape(d_up.shape[0], d_up.shape[1] // 2, 2, d_up.shape[2] // 2, 2).sum(axis=(2, 4))",
                               "da = d_up.reshape(d_up.shape[0], d_up.shape[1] // 2, 2, d_up.shape[2] // 2, 2).mean(axis=(2, 4))"),
}


@pytest.mark.parametrize("name", sorted(GRAD_MUTANTS))
def test_gradient_pin_catches_mutant(name, tmp_path):
    import shutil

    old, new = GRAD_MUTANTS[name]
    src = open(UNET).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    (tmp_path / "oracle" / "unet.py").write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=f"{tmp_path}{os.pathsep}{ROOT}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_unet_grad.py") + "::test_gradient_matches_finite_differences"],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed the gradient pin:\n{r.stdout[-2000:]}"
