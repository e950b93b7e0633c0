"""Tensor-core layers of the learned inpainter against its CPU definition (oracle/unet.py),
through the C ABI (needs a GPU).

A tcgen05 convolution sums the BF16 products in another order than the definition
(input channel, kernel row, kernel column), so the two agree within the error bound of
FP32 summation, not bit for bit.  For an output whose products are p_i (exact in FP32:
a product of two bfloat16 values has at most 16 significant bits), the definition's
sequential sum is within K u sum |p_i| of the exact sum (u = 2^-24, K products); the
tensor core's accumulation is allowed twice that (one unit in the last place per
addition).  So before rounding |gpu - oracle| <= 3 K u sum |p_i| + the bias addition's
rounding; after ReLU and rounding to bfloat16 the two may also land one bfloat16 step
apart where the value sits next to a rounding boundary.  The test allows exactly that
per element: tol = 3 K u sum|p| (1 + 2^-7) + 2 ulp_f32(|o|) + ulp_bf16(max(|o|, |g|)).
"""
import numpy as np
import pytest
import torch

from oracle import unet as ref

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def un():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_15183_gb300 as yoro
    from paper_2506_15183_gb300 import _build
    from paper_2506_15183_gb300 import unet

    _build.build_cuda()
    yoro.load_library()
    return unet


def _bf16_t(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()


def _ulp_bf16(v):
    v = np.maximum(np.abs(v), np.float32(2.0 ** -126))
    return np.exp2(np.floor(np.log2(v)) - 7).astype(np.float64)


def _case(un, T, H, W, cin, cout, seed, upsample=False, cy=None, coff=0, relu=True, real_cin=None):
    rng = np.random.default_rng(seed)
    real_cin = real_cin or cin
    x = np.zeros((T, real_cin, H, W), np.float32)
    x[:] = ref.bf16(rng.uniform(0.0, 1.0, x.shape).astype(np.float32))
    w = ref.bf16(rng.normal(0.0, np.sqrt(2.0 / (9 * real_cin)), (cout, real_cin, 3, 3)).astype(np.float32))
    b = rng.normal(0.0, 0.05, cout).astype(np.float32)
    # GPU: NHWC with Cin padded to a multiple of 32
    xp = np.zeros((T, H, W, cin), np.float32)
    xp[..., :real_cin] = np.transpose(x, (0, 2, 3, 1))
    cy = cy or cout
    f = 2 if upsample else 1
    y = torch.full((T, f * H, f * W, cy), 7.0, dtype=torch.bfloat16, device="cuda")
    wk = un.kmajor(w)
    if wk.shape[1] != 9 * cin:
        wk2 = np.zeros((cout, 9 * cin), np.float32)
        wk3 = wk.reshape(cout, 9, -1)
        wk2.reshape(cout, 9, cin)[:, :, :wk3.shape[2]] = wk3
        wk = wk2
    un.conv3x3(_bf16_t(xp), _bf16_t(wk), torch.from_numpy(b).cuda(), y, y_coff=coff, upsample=upsample, relu=relu)
    assert un.status() == 0
    g = y.float().cpu().numpy()
    for t in range(T):
        pre = ref.conv3x3(x[t], w, b)
        o = ref.relu_bf16(pre) if relu else ref.bf16(pre)
        absum = ref.conv3x3(np.abs(x[t]), np.abs(w), np.zeros(cout, np.float32)).astype(np.float64)
        K = 9 * real_cin
        go = g[t][..., coff:coff + cout]
        if upsample:
            for a in (0, 1):
                for c in (0, 1):
                    _compare(go[a::2, c::2].transpose(2, 0, 1), o, absum, K)
        else:
            _compare(go.transpose(2, 0, 1), o, absum, K)
        # channels outside [coff, coff + cout) are untouched
        if cy > cout:
            rest = np.delete(g[t], np.arange(coff, coff + cout), axis=-1)
            assert np.all(rest == 7.0)


def _compare(g, o, absum, K):
    o64, g64 = o.astype(np.float64), g.astype(np.float64)
    tol = 3 * K * U * absum * (1 + 2.0 ** -7) + 2 * np.abs(o64) * 2.0 ** -23 + _ulp_bf16(np.maximum(np.abs(o), np.abs(g)))
    bad = np.abs(g64 - o64) > tol
    assert not bad.any(), f"{bad.sum()} of {bad.size} outside the bound; worst {np.abs(g64 - o64)[bad].max()}"
    assert np.mean(g64 != o64) < 0.05  # almost every element is the same bfloat16 value


@pytest.mark.parametrize("T,H,W,cin,cout", [(1, 64, 64, 32, 32), (2, 32, 32, 32, 64), (1, 16, 16, 64, 128),
                                              (2, 8, 8, 128, 256), (3, 16, 16, 384, 128), (1, 64, 64, 96, 32)])
def test_conv_layer_matches_definition(un, T, H, W, cin, cout):
    _case(un, T, H, W, cin, cout, seed=100 + cin + cout)


def test_conv_first_layer_padded_channels(un):
    """The 6 input channels padded to 32 with zero channels and zero weights."""
    _case(un, 1, 64, 64, 32, 32, seed=7, real_cin=6)


def test_conv_into_concat_buffer_and_upsampled(un):
    """Channel offset inside a wider buffer, and the 2x2 nearest-upsampling store."""
    _case(un, 2, 8, 8, 256, 256, seed=8, upsample=True, cy=384, coff=128)
    _case(un, 1, 32, 32, 64, 32, seed=9, cy=96, coff=0)


def test_conv_without_relu(un):
    _case(un, 1, 16, 16, 64, 64, seed=10, relu=False)
