"""Oracle of the learned warm start -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this module.  It is plain numpy in float64 and
shares no code with the CUDA path.

The paper starts its iteration from an unspecified point (Section 3; the cold
start lambda = 0 is the reading used by the solver).  The warm start predicts a
starting lambda from each node's neighbourhood, and GDP then runs exactly as
from any other start, so the prediction only changes where the iteration
begins, never what it certifies.

Definitions followed here and by the CUDA kernels:

* features of node v: the distances to its 16 nearest other points (exact
  int64 squared distances, ties by index), ascending, divided by
  s_v = max(1, mean of those 16 distances);
* network: 16 -> 128 -> 128 -> 1, ReLU after the two hidden layers; its output
  predicts lambda_v / s_v (lambda in length units);
* arithmetic: the inputs of every matrix product on the tensor cores are
  rounded to bfloat16 (round to nearest even) -- the features, W1, W2, the
  first hidden activations, and in the backward pass the gradients at the two
  hidden pre-activations, the second hidden activations and dL/dy -- and the
  products are accumulated in float32 (here: float64);
* loss: mean squared error over the samples of a step; optimiser: Adam;
* warm start: lambda0_v = rint(2^F * s_v * y_v), clamped to |lambda0| <= 2^27.

Parameter vector layout (float32 [18817]): W1 [128][16] (output-major), b1
[128], W2 [128][128], b2 [128], w3 [128], b3 [1].
"""
from __future__ import annotations

import numpy as np

K_FEAT = 16
H = 128
NPARAMS = H * K_FEAT + H + H * H + H + H + 1
LAMBDA0_LIMIT = 1 << 27


def unpack(params):
    """Views of the flat parameter vector: (W1, b1, W2, b2, w3, b3)."""
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * K_FEAT].reshape(H, K_FEAT); o += H * K_FEAT
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, np.atleast_1d(b3)]).astype(np.float64)


def bf16(x):
    """Round to the nearest bfloat16 (8 significant bits), ties to even; the
    result is returned as float64.  Finite inputs within the float32 range."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)               # x = m * 2^e, 0.5 <= |m| < 1
    q = np.rint(m * 256.0)           # 8 significant bits; np.rint ties to even
    return np.ldexp(q / 256.0, e)


def features(d2):
    """(feat [n][16] float64, s [n] float64) from the squared distances to the 16
    nearest neighbours, each row ascending."""
    dist = np.sqrt(np.asarray(d2, dtype=np.float64))
    s = np.maximum(1.0, dist.mean(axis=1))
    return dist / s[:, None], s


def forward(params, feat, rounding=True):
    """Network output y [B] and the intermediates the backward pass needs."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(params)
    f = r(feat)
    z1 = f @ r(W1).T + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(W2).T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, dict(f=f, z1=z1, h1=h1, z2=z2, h2=h2)


def backward(params, feat, target, rounding=True):
    """(loss, gradient [NPARAMS]) of loss = mean_b (y_b - t_b)^2 over the B samples."""
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(params)
    y, c = forward(params, feat, rounding)
    t = np.asarray(target, dtype=np.float64)
    B = y.shape[0]
    res = y - t
    loss = float(np.mean(res * res))
    dy = 2.0 * res / B
    g_b3 = dy.sum()
    g_w3 = r(c["h2"]).T @ r(dy)
    dz2 = r(dy[:, None] * w3[None, :] * (c["z2"] > 0))
    g_W2 = dz2.T @ c["h1"]
    g_b2 = dz2.sum(axis=0)
    dh1 = dz2 @ r(W2)
    dz1 = r(dh1 * (c["z1"] > 0))
    g_W1 = dz1.T @ c["f"]
    g_b1 = dz1.sum(axis=0)
    return loss, pack(g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)


def adam(params, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) with bias correction; ``step`` counts
    from 1.  Returns new (params, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p = np.asarray(params, dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def warm_lambda(y, s, F=8):
    """lambda0 in units 2^-F from the network output y = lambda / s."""
    lam = np.rint(np.ldexp(np.asarray(s, dtype=np.float64) * np.asarray(y, dtype=np.float64), F))
    return np.clip(lam, -LAMBDA0_LIMIT, LAMBDA0_LIMIT).astype(np.int32)
