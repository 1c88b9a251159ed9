"""The learned block proposal's tensor-core kernels (tcgen05, BF16 operands, FP32 accumulation)
against the CPU oracle oracle/cnn.py, through the C-ABI.

The oracle rounds to BF16 at the same points as the kernels (input features, conv weights, stored
activations and activation gradients) and sums in FP64, so the two differ by accumulation order
and by the few values that land on the other side of a BF16 rounding boundary: probabilities
within 5e-3 (mean 5e-4), each layer's gradient within 3 % in norm, the loss within 1e-3."""
import numpy as np
import pytest

from oracle import cnn as C
from paper_2103_07417_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    yield c
    c.close()


def _params(seed):
    p = W.cnn_init(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    u = C.unpack(p)
    for k in ("b1", "b2", "b3", "b4"):
        u[k][:] = rng.normal(0, 0.05, u[k].shape)
    u["bh"][:] = -0.3
    return C.pack(u).astype(np.float32)


def _features(seed, H, Wd):
    rng = np.random.default_rng(seed)
    f = np.stack([np.arcsinh(np.exp(rng.normal(-1, 1.5, (H, Wd)))),
                  3.0 / np.maximum(rng.uniform(1, 40, (H, Wd)), 1.0),
                  rng.integers(0, 3, (H, Wd)).astype(float)], -1)
    return f.astype(np.float32)


@pytest.mark.parametrize("H,Wd", [(37, 29), (9, 9), (129, 65), (1, 7)])
def test_cnn_forward_matches_oracle(ctx, H, Wd):
    prm = _params(1)
    ctx.art_cnn_load(prm)
    f = _features(H * 7 + Wd, H, Wd)
    p_gpu = ctx.art_cnn_forward(torch.from_numpy(f).cuda()).cpu().numpy()
    _, _, p_ref = C.forward(prm.astype(np.float64), f.astype(np.float64), quantize=True)
    assert p_gpu.shape == p_ref.shape == (C.head_size(H), C.head_size(Wd))
    d = np.abs(p_gpu - p_ref)
    assert d.max() < 5e-3 and d.mean() < 5e-4, (d.max(), d.mean())


@pytest.mark.parametrize("H,Wd", [(37, 29), (65, 65)])
def test_cnn_gradients_match_oracle(ctx, H, Wd):
    prm = _params(2)
    ctx.art_cnn_load(prm)
    f = _features(H + 3 * Wd, H, Wd)
    rng = np.random.default_rng(5)
    t = (rng.uniform(size=(C.head_size(H), C.head_size(Wd))) < 0.3).astype(np.float32)
    loss, g = ctx.art_cnn_grad(torch.from_numpy(f).cuda(), torch.from_numpy(t).cuda())
    loss_ref, g_ref = C.loss_and_grad(prm.astype(np.float64), f.astype(np.float64), t, quantize=True)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    off = 0
    for name, shp in C.SHAPES:
        n = int(np.prod(shp))
        a, b = g[off:off + n].astype(np.float64), g_ref[off:off + n]
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert err < 3e-2, (name, err)
        # element by element: the BF16 rounding points are the oracle's too, so an element
        # differs only by FP32-vs-FP64 summation and the activations whose BF16 rounding that
        # moves by one ulp (2^-8 relative); bounded by a small fraction of the layer's largest
        # gradient plus a few BF16 ulps of the element itself
        big = np.abs(b).max()
        worst = np.max(np.abs(a - b) / (big + 1e-30))
        print(name, "max |dg| / max|g|", worst)
        assert np.all(np.abs(a - b) <= 5e-3 * big + 4 * 2.0 ** -8 * np.abs(b)), (name, worst)
        off += n


def test_cnn_training_reduces_loss(ctx):
    """Adam on a fixed lattice: the tensor-core forward/backward drives the loss down."""
    ctx.art_cnn_load(_params(3))
    f = _features(11, 65, 65)
    yy, xx = np.mgrid[0:C.head_size(65), 0:C.head_size(65)]
    t = (np.hypot(yy - 8, xx - 8) < 5).astype(np.float32)   # a disc of positive blocks
    fd, td = torch.from_numpy(f).cuda(), torch.from_numpy(t).cuda()
    first = ctx.art_cnn_train_step(fd, td, 3e-3)
    for _ in range(150):
        last = ctx.art_cnn_train_step(fd, td, 3e-3)
    assert last < 0.5 * first, (first, last)
    back = ctx.art_cnn_read()
    assert np.isfinite(back).all()
