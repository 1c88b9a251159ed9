"""Pins of the oracle of the learned block proposal (oracle/cnn.py).

The network is not in the paper; its oracle is pinned to library routines and exact identities:
each 3x3 convolution against scipy's 2-D correlation, the stride-2 convolution against every
other output of the stride-1 one, BF16 rounding against torch's conversion, the output size of the
two stride-2 stages, the cross-entropy against its definition, and the whole backward pass against
central finite differences of the loss (FP64, no rounding)."""
import numpy as np
import pytest

from oracle import cnn as C
from paper_2103_07417_gb300 import workloads as W

signal = pytest.importorskip("scipy.signal")
torch = pytest.importorskip("torch")


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((11, 9, 3))
    Wt = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = C.conv3x3(x, Wt, b, 1)
    for co in range(4):
        ref = sum(signal.correlate2d(x[:, :, ci], Wt[co, :, :, ci], mode="same") for ci in range(3))
        np.testing.assert_allclose(y[:, :, co], ref + b[co], rtol=1e-12, atol=1e-12)


def test_stride_two_is_every_other_output():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((13, 10, 5))
    Wt = rng.standard_normal((6, 3, 3, 5))
    b = rng.standard_normal(6)
    np.testing.assert_allclose(C.conv3x3(x, Wt, b, 2), C.conv3x3(x, Wt, b, 1)[::2, ::2], rtol=1e-12)
    assert C.head_size(129) == 33 and C.head_size(2049) == 513 and C.head_size(10) == 3


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.uniform(-30, 30, 2000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 3.3895e38]])
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(C.bf16(v), ref)


def test_bce_definition():
    z = np.array([[-3.0, 0.0], [2.0, 15.0]])
    t = np.array([[0.0, 1.0], [1.0, 0.0]])
    p = 1 / (1 + np.exp(-z))
    ref = -np.mean(t * np.log(p) + (1 - t) * np.log1p(-p))
    assert C.bce(z, t) == pytest.approx(ref, rel=1e-9)   # the direct form loses ~1e-11 at z = 15


def test_backward_matches_finite_differences():
    """Every parameter gradient of the full network (FP64, no rounding) against central
    differences of the loss, on a 13 x 11 lattice; a random subset of 400 weights plus all biases
    and the head."""
    params = W.cnn_init(3).astype(np.float64)
    params[C.N_PARAMS - 33:] += 0.1   # move the head off zero so every path carries gradient
    rng = np.random.default_rng(4)
    x = rng.standard_normal((13, 11, 3))
    t = (rng.uniform(size=(C.head_size(13), C.head_size(11))) < 0.4).astype(np.float64)
    loss, g = C.loss_and_grad(params, x, t, quantize=False)
    assert np.isfinite(loss)
    idx = np.concatenate([rng.choice(C.N_PARAMS - 33 - 128, 400, replace=False),
                          np.arange(C.N_PARAMS - 33, C.N_PARAMS)])
    off = 0
    bias_idx = []
    for name, shp in C.SHAPES:
        n = int(np.prod(shp))
        if name.startswith("b"):
            bias_idx.extend(range(off, off + n))
        off += n
    idx = np.unique(np.concatenate([idx, bias_idx]))
    h = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (C.loss_and_grad(pp, x, t, quantize=False)[0] - C.loss_and_grad(pm, x, t, quantize=False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_features_of_a_level():
    img = np.arange(81.0).reshape(9, 9)
    mr = np.full((9, 9), 0.5)
    mr[0, 0] = 6.0
    nt = np.ones((9, 9))
    f = C.features(img, mr, nt, 2.0, 1, 3)          # stride 4 lattice: 3 x 3
    assert f.shape == (3, 3, 3)
    assert f[0, 1, 0] == pytest.approx(np.arcsinh(4.0 / 2.0))
    assert f[0, 0, 1] == pytest.approx(0.5) and f[1, 1, 1] == pytest.approx(3.0)
