"""Pins of the learned-warm-start oracle (oracle/learned.py, or_knn) against
things other than itself: a library bfloat16 conversion, a k-d tree, the
independent input builder, PyTorch autograd, finite differences and closed
forms of Adam's first steps."""
import numpy as np
import pytest

import instances as I
import oracle
from oracle import learned as L


# ---- bfloat16 rounding --------------------------------------------------------------

def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(200000).astype(np.float32) * np.float32(3.0),
        rng.uniform(-1e-3, 1e-3, 20000).astype(np.float32),
        np.float32(1.0) + np.arange(-512, 512, dtype=np.float32) * np.float32(2.0 ** -9),
    ])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16(x.astype(np.float64)), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: the even neighbour is 1
    assert L.bf16(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    assert L.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert L.bf16(-(1.0 + 2.0 ** -8)) == -1.0
    assert L.bf16(255.5) == 256.0 and L.bf16(254.5) == 254.0


# ---- k nearest neighbours -----------------------------------------------------------

def test_knn_distances_match_kdtree():
    cKDTree = pytest.importorskip("scipy.spatial").cKDTree
    xy = I.mixture_points(3000, 5)
    nbr, d2 = oracle.knn(xy, 16)
    dist, _ = cKDTree(xy.astype(np.float64)).query(xy.astype(np.float64), k=17)
    # the k-d tree includes the point itself (or a copy at distance 0) first
    ref = np.rint(dist[:, 1:] ** 2).astype(np.int64)
    assert np.array_equal(d2, ref)
    # listed distances agree with the listed indices
    d = xy[nbr].astype(np.int64) - xy[:, None, :].astype(np.int64)
    assert np.array_equal(d2, d[..., 0] ** 2 + d[..., 1] ** 2)


def test_knn_ties_by_index_brute_force():
    # a 6x6 unit grid has ties at every distance; add two copies of one point
    g = np.array([(i, j) for i in range(6) for j in range(6)], dtype=np.int32)
    xy = np.concatenate([g, g[[7, 7]]])
    k = 9
    nbr, d2 = oracle.knn(xy, k)
    for i in range(xy.shape[0]):
        cand = sorted(((int(xy[j, 0]) - int(xy[i, 0])) ** 2 + (int(xy[j, 1]) - int(xy[i, 1])) ** 2, j)
                      for j in range(xy.shape[0]) if j != i)[:k]
        assert [c[1] for c in cand] == nbr[i].tolist()
        assert [c[0] for c in cand] == d2[i].tolist()


@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 2500, 1, 10), ("mixture", 3000, 2, 12),
                                           ("uniform", 40, 3, 3)])
def test_knn_csr_matches_input_builder(kind, n, seed, k):
    d = I.make_instance(kind, n, seed, k)
    rp, col = oracle.knn_csr(d["xy"], k)
    assert np.array_equal(rp, d["row_ptr"]) and np.array_equal(col, d["col"])


# ---- features -----------------------------------------------------------------------

def test_features_closed_form():
    # 17 points on a line at x = 0, 1, 3, 6, ... : point 0's neighbours are at
    # the triangular numbers T_1..T_16, mean 816/16 = 51
    xs = np.array([j * (j + 1) // 2 for j in range(17)], dtype=np.int64)
    xy = np.stack([xs, np.zeros_like(xs)], axis=1).astype(np.int32)
    _, d2 = oracle.knn(xy, 16)
    f, s = L.features(d2)
    assert s[0] == 51.0
    assert np.allclose(f[0], xs[1:] / 51.0, rtol=0, atol=1e-15)
    # scale invariance: features do not change when coordinates scale by 7
    _, d2b = oracle.knn(xy * 7, 16)
    fb, sb = L.features(d2b)
    assert np.allclose(fb, f, rtol=1e-14) and np.allclose(sb, 7 * s)


def test_features_scale_floor():
    # 17 copies of one point: every distance 0, s = max(1, 0) = 1, features 0
    xy = np.zeros((17, 2), dtype=np.int32)
    _, d2 = oracle.knn(xy, 16)
    f, s = L.features(d2)
    assert np.all(s == 1.0) and np.all(f == 0.0)


# ---- network: forward and backward --------------------------------------------------

def _batch(B, seed):
    feat = I.uniform_floats(seed, B * 16, 0.2, 2.5).reshape(B, 16).astype(np.float64)
    feat.sort(axis=1)
    target = I.uniform_floats(seed + 1, B, 0.2, 0.6).astype(np.float64)
    return feat, target


def test_backward_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    p = I.mlp_init(3).astype(np.float64)
    feat, target = _batch(64, 11)
    loss, g = L.backward(p, feat, target, rounding=False)
    P = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    o = 0
    W1 = P[o:o + 2048].view(128, 16); o += 2048
    b1 = P[o:o + 128]; o += 128
    W2 = P[o:o + 16384].view(128, 128); o += 16384
    b2 = P[o:o + 128]; o += 128
    w3 = P[o:o + 128]; o += 128
    b3 = P[o]
    x = torch.tensor(feat)
    y = torch.relu(torch.relu(x @ W1.T + b1) @ W2.T + b2) @ w3 + b3
    lt = torch.mean((y - torch.tensor(target)) ** 2)
    lt.backward()
    assert abs(loss - lt.item()) < 1e-12
    assert np.allclose(g, P.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_backward_matches_finite_differences():
    p = I.mlp_init(4).astype(np.float64)
    feat, target = _batch(32, 21)
    _, g = L.backward(p, feat, target, rounding=False)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(2048, 6, replace=False), 2048 + rng.choice(128, 3, replace=False),
                          2176 + rng.choice(16384, 6, replace=False), 18560 + rng.choice(128, 3, replace=False),
                          18688 + rng.choice(128, 3, replace=False), [18816]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp = np.mean((L.forward(p + e, feat, False)[0] - target) ** 2)
        lm = np.mean((L.forward(p - e, feat, False)[0] - target) ** 2)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_rounded_forward_close_to_exact():
    # bfloat16 inputs change the output by a few parts in 2^8 at most
    p = I.mlp_init(5).astype(np.float64)
    feat, _ = _batch(256, 31)
    y0, _ = L.forward(p, feat, rounding=False)
    y1, _ = L.forward(p, feat, rounding=True)
    assert np.max(np.abs(y1 - y0)) < 0.05 * np.max(np.abs(y0)) and not np.array_equal(y0, y1)


def test_forward_hand_example():
    # one path through the network: y = w3[5] * relu(W2[5,2] * relu(W1[2,0] f0 + b1[2]) + b2[5]) + b3
    W1 = np.zeros((128, 16)); b1 = np.zeros(128); W2 = np.zeros((128, 128)); b2 = np.zeros(128)
    w3 = np.zeros(128)
    W1[2, 0] = 2.0; b1[2] = -0.5; W2[5, 2] = 3.0; b2[5] = 0.25; w3[5] = -1.5; b3 = 0.125
    p = L.pack(W1, b1, W2, b2, w3, b3)
    feat = np.zeros((2, 16)); feat[0, 0] = 1.0; feat[1, 0] = 0.125
    y, _ = L.forward(p, feat, rounding=True)
    # sample 0: z1 = 1.5, h1 = 1.5, z2 = 4.75, y = -7.125 + 0.125 = -7.0
    # sample 1: z1 = -0.25 -> h1 = 0, z2 = 0.25, y = -0.375 + 0.125 = -0.25
    assert y.tolist() == [-7.0, -0.25]
    loss, g = L.backward(p, feat, np.array([-6.0, 0.0]), rounding=True)
    # residuals -1 and -0.25: loss = (1 + 1/16) / 2, dy = residual
    assert loss == (1.0 + 0.0625) / 2
    gW1, gb1, gW2, gb2, gw3, gb3 = L.unpack(g)
    assert gb3 == -1.25
    assert gw3[5] == -1.0 * 4.75 + -0.25 * 0.25
    # dz2[., 5] = dy * w3[5] = 1.5 and 0.375; dW2[5, 2] = 1.5 * h1 = 2.25
    assert gb2[5] == 1.875 and gW2[5, 2] == 2.25
    # dz1[0, 2] = dz2[0, 5] * W2[5, 2] = 4.5 (sample 1 is cut by the ReLU)
    assert gb1[2] == 4.5 and gW1[2, 0] == 4.5
    assert np.count_nonzero(g) == 6


# ---- Adam ---------------------------------------------------------------------------

def test_adam_first_steps_closed_form():
    p0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    p1, m, v = L.adam(p0, np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    # after bias correction the first step is lr * g / (|g| + eps)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    p2, _, _ = L.adam(p1, m, v, g, 2, lr=0.01)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    assert np.allclose(p2, p0 - 0.02 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_warm_lambda_rounding_and_clamp():
    s = np.array([1.0, 1.0, 2.0, 1.0, 1e6])
    y = np.array([0.5 / 256, 1.5 / 256, 0.25, -2.5 / 256, 1e6])
    lam = L.warm_lambda(y, s, F=8)
    assert lam.tolist() == [0, 2, 128, -2, 1 << 27]
