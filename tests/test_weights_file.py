"""The inpainter's parameter table and weights file (host only)."""
import numpy as np
import pytest

from oracle import unet as ref
from paper_2506_15183_gb300 import weights as W


def test_layer_table_matches_the_definition():
    got = [(n, tuple(ws), nb) for n, ws, nb in W.layers()]
    want = [(n, tuple(ws), bs[0]) for n, ws, bs in ref.layer_shapes()]
    assert got == want


def test_flops_per_tile():
    # 2 x multiply-adds of every layer at its level's side, counted independently
    want = 0
    for n, ws, _ in ref.layer_shapes():
        side = 64 if n == "out" else 64 >> int(n[3])
        want += 2 * side * side * int(np.prod(ws))
    assert W.flops_per_tile() == want
    assert abs(W.flops_per_tile() / 1.34e9 - 1) < 0.01


def test_round_trip_and_refusals(tmp_path):
    p = W.init_params(3)
    f = str(tmp_path / "u.yw")
    W.save(p, f, steps=5, ktiles=7, loss=0.25, seed=3)
    q, meta = W.read(f)
    assert np.array_equal(p, q) and meta == dict(steps=5, ktiles=7, loss=0.25, seed=3)
    raw = bytearray(open(f, "rb").read())
    for mutate in (lambda b: b.__setitem__(0, ord("X")),      # magic
                   lambda b: b.__setitem__(4, 2),             # version
                   lambda b: b.__setitem__(40, b[40] ^ 1)):   # a parameter byte: checksum
        bad = bytearray(raw)
        mutate(bad)
        open(f, "wb").write(bad)
        with pytest.raises(ValueError):
            W.read(f)
    with pytest.raises(ValueError):
        W.save(p[:-1], f)


def test_split_views_every_parameter_once():
    p = np.arange(W.count(), dtype=np.float32)
    parts = W.split(p)
    cat = np.concatenate([np.concatenate([parts[n + ".w"].ravel(), parts[n + ".b"]]) for n, _, _ in W.layers()])
    assert np.array_equal(cat, p)
