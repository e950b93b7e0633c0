"""The inpainter's loss gradient (oracle/unet.py loss_and_grads) against finite
differences of the loss, in float64 with no bfloat16 rounding, on a 16 x 16 tile (the
network is fully convolutional; 16 x 16 reaches the 2 x 2 bottom level).  A missing
term, a transposed or unflipped kernel, a gradient sent to the wrong pooling input or
concatenation half would each fail it."""
import numpy as np

from oracle import unet as ref


def _setup(seed, side=16):
    rng = np.random.default_rng(seed)
    p = ref.init_weights(seed)
    p = {k: v.astype(np.float64) for k, v in p.items()}
    for name, _, bs in ref.layer_shapes():
        p[name + ".b"] = rng.normal(0.0, 0.1, bs)
    x = rng.uniform(0.0, 1.0, (6, side, side))
    gt = rng.uniform(0.0, 1.0, (3, side, side))
    hole = rng.uniform(size=(side, side)) < 0.4
    return p, x, gt, hole


def test_gradient_matches_finite_differences():
    p, x, gt, hole = _setup(5)
    loss, g = ref.loss_and_grads(x, p, gt, hole, exact=True)
    rng = np.random.default_rng(9)
    eps = 1e-6
    for name, ws, bs in ref.layer_shapes():
        for key, shape in ((name + ".w", ws), (name + ".b", bs)):
            for _ in range(3):
                idx = tuple(int(rng.integers(0, d)) for d in shape)
                q = {k: v.copy() for k, v in p.items()}
                q[key][idx] += eps
                lp, _ = ref.loss_and_grads(x, q, gt, hole, exact=True)
                q[key][idx] -= 2 * eps
                lm, _ = ref.loss_and_grads(x, q, gt, hole, exact=True)
                fd = (lp - lm) / (2 * eps)
                an = g[key][idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (key, idx, fd, an)


def test_bf16_forward_gradient_is_close_to_exact():
    """With the definition's bfloat16 forward the gradient moves only by the rounding's
    effects (a ReLU or pooling decision that flips, activations one bfloat16 step off):
    measured up to 17 % relative L2 in the deepest layers of this 16 x 16 tile, whose
    bottom level has 2 x 2 pixels; the bound is 25 % with cosine >= 0.98 per tensor."""
    p, x, gt, hole = _setup(6)
    _, g64 = ref.loss_and_grads(x, p, gt, hole, exact=True)
    _, g16 = ref.loss_and_grads(x, p, gt, hole, exact=False)
    for k in g64:
        a, b = g64[k].ravel(), g16[k].ravel()
        assert np.linalg.norm(a - b) <= 0.25 * np.linalg.norm(a) + 1e-12, k
        assert np.dot(a, b) >= 0.98 * np.linalg.norm(a) * np.linalg.norm(b), k
