"""TEST INFRASTRUCTURE ONLY: CPU oracle of the learned block proposal (the CNN of the adaptive
ray tracer's learned path).

The paper has no learned component; the proposal network is an addition whose only job is to
predict, from the completed level-k lattice, which blocks the exact criterion of Sec. 3.2 will
refine two levels later, so those rays can be traced early.  The exact criterion still decides
every point.  This module is the plain reference the GPU kernels are checked against:

    features  f0 = asinh(I / (R_abs I_norm)), f1 = 3 / max(r_min, 1), f2 = polar turns, on the
              level-k lattice (stride 2^(N-k) of the final grid); I_norm = the criterion's
              normalisation, R_abs its absolute tolerance (I_norm alone when R_abs <= 0; f0 = 0
              when that scale is not positive).
    c1  3x3 conv,  3 -> 32, stride 1, pad 1, + bias, ReLU
    c2  3x3 conv, 32 -> 32, stride 1, pad 1, + bias, ReLU
    c3  3x3 conv, 32 -> 32, stride 2, pad 1, + bias, ReLU
    c4  3x3 conv, 32 -> 32, stride 2, pad 1, + bias, ReLU
    head  1x1 conv 32 -> 1 + bias, logistic sigmoid: one probability per 4 x 4 lattice cells
    loss  mean binary cross-entropy against 0/1 block labels.

Arithmetic: FP64 sums.  With quantize=True the values the GPU keeps in BF16 are rounded to BF16
at the same points (the input features, the conv weights, every stored activation and every
stored activation gradient); weights of the head, biases, logits and all gradient sums stay
unrounded.  Convolutions are written as im2col + matrix product (a library primitive).
Parameter vector (FP32, in this order): W1 (32, 3, 3, 3), b1 (32), W2 (32, 3, 3, 32), b2, W3, b3,
W4, b4, w_head (32), b_head (1); conv weights indexed [out][ky][kx][in].

Pinned by tests/test_oracle_cnn.py (convolution against scipy's correlate2d, the stride-2 identity,
BF16 rounding against torch's conversion, backward against central finite differences).
"""
from __future__ import annotations

import numpy as np

CH = 32
SHAPES = [("W1", (CH, 3, 3, 3)), ("b1", (CH,)), ("W2", (CH, 3, 3, CH)), ("b2", (CH,)),
          ("W3", (CH, 3, 3, CH)), ("b3", (CH,)), ("W4", (CH, 3, 3, CH)), ("b4", (CH,)),
          ("wh", (CH,)), ("bh", (1,))]
STRIDES = (1, 1, 2, 2)
N_PARAMS = int(sum(np.prod(s) for _, s in SHAPES))


def unpack(vec) -> dict:
    vec = np.asarray(vec, dtype=np.float64).ravel()
    if vec.size != N_PARAMS:
        raise ValueError(f"expected {N_PARAMS} parameters")
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = vec[o:o + n].reshape(shp)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(nan, np.nan, out)


def out_size(n: int, stride: int) -> int:
    """Output length of a 3-tap, pad-1 convolution: floor((n - 1)/stride) + 1."""
    return (n - 1) // stride + 1


def head_size(n: int) -> int:
    return out_size(out_size(n, 2), 2)


def features(img, min_r, nturn, norm: float, level: int, levels: int, r_abs: float = 0.0):
    """(H, W, 3) features of the level-`level` lattice of final-resolution planes."""
    if r_abs > 0:
        norm = norm * r_abs
    s = 1 << (levels - level)
    I = np.asarray(img, dtype=np.float64)[::s, ::s]
    mr = np.asarray(min_r, dtype=np.float64)[::s, ::s]
    nt = np.asarray(nturn, dtype=np.float64)[::s, ::s]
    f0 = np.arcsinh(I / norm) if norm > 0 else np.zeros_like(I)   # a dark image gives 0
    return np.stack([f0, 3.0 / np.maximum(mr, 1.0), nt], axis=-1)


def _im2col(x, stride):
    """(Ho*Wo, 9*C) patches of a zero-padded 3x3 window, columns ordered (ky, kx, c)."""
    H, W, C = x.shape
    Ho, Wo = out_size(H, stride), out_size(W, stride)
    xp = np.zeros((H + 2, W + 2, C))
    xp[1:-1, 1:-1] = x
    cols = np.empty((Ho, Wo, 3, 3, C))
    for ky in range(3):
        for kx in range(3):
            cols[:, :, ky, kx, :] = xp[ky:ky + stride * (Ho - 1) + 1:stride,
                                       kx:kx + stride * (Wo - 1) + 1:stride]
    return cols.reshape(Ho * Wo, 9 * C), (Ho, Wo)


def conv3x3(x, W, b, stride):
    """y[o] = b + sum over (ky, kx, c) of W[:, ky, kx, c] x[stride*o + (ky, kx) - 1, c]."""
    cols, (Ho, Wo) = _im2col(np.asarray(x, dtype=np.float64), stride)
    Wm = np.asarray(W, dtype=np.float64).reshape(W.shape[0], -1)
    return (cols @ Wm.T + b).reshape(Ho, Wo, W.shape[0])


def _col2im(dcols, shape, stride):
    """Adjoint of _im2col: scatter-add patch gradients back onto the input grid."""
    H, W, C = shape
    Ho, Wo = out_size(H, stride), out_size(W, stride)
    d = dcols.reshape(Ho, Wo, 3, 3, C)
    dxp = np.zeros((H + 2, W + 2, C))
    for ky in range(3):
        for kx in range(3):
            dxp[ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride] += d[:, :, ky, kx, :]
    return dxp[1:-1, 1:-1]


def forward(params, x, quantize: bool = True):
    """Activations (list of the four stored conv outputs), logits and probabilities."""
    p = unpack(params) if not isinstance(params, dict) else params
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    h = q(x)
    acts = [h]
    for i, s in enumerate(STRIDES):
        Wq = q(p[f"W{i + 1}"])
        h = q(np.maximum(conv3x3(h, Wq, p[f"b{i + 1}"], s), 0.0))
        acts.append(h)
    logits = acts[-1] @ p["wh"] + p["bh"][0]
    return acts, logits, 1.0 / (1.0 + np.exp(-logits))


def bce(logits, target):
    """Mean binary cross-entropy of sigmoid(logits) against 0/1 targets (stable form)."""
    z = np.asarray(logits, dtype=np.float64)
    t = np.asarray(target, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0) - z * t + np.log1p(np.exp(-np.abs(z)))))


def loss_and_grad(params, x, target, quantize: bool = True):
    """BCE loss and the gradient of every parameter (packed like the parameter vector)."""
    p = unpack(params) if not isinstance(params, dict) else params
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    acts, logits, prob = forward(p, x, quantize)
    t = np.asarray(target, dtype=np.float64)
    n = t.size
    loss = bce(logits, t)
    dlog = (prob - t) / n
    g = {"wh": np.tensordot(dlog, acts[-1], axes=([0, 1], [0, 1])), "bh": np.array([dlog.sum()])}
    # gradient at the stored output of c4, through its ReLU
    dy = q(dlog[..., None] * p["wh"][None, None, :] * (acts[-1] > 0))
    for i in range(3, -1, -1):
        s = STRIDES[i]
        xin = acts[i]
        Wq = q(p[f"W{i + 1}"])
        cols, _ = _im2col(xin, s)
        dyf = dy.reshape(-1, dy.shape[-1])
        g[f"W{i + 1}"] = (dyf.T @ cols).reshape(Wq.shape)
        g[f"b{i + 1}"] = dyf.sum(axis=0)
        if i > 0:
            dx = _col2im(dyf @ Wq.reshape(Wq.shape[0], -1), xin.shape, s)
            dy = q(dx * (xin > 0))
    return loss, pack(g)
