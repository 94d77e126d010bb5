"""Seeded synthetic F2M instances: integer point sets and k-nearest-neighbour CSRs.

This module is the only code that the CPU oracle and the CUDA path share.  It
draws points and builds the candidate graph that both sides receive as input;
it holds none of the method's arithmetic (no edge cost, no reduced cost, no
dual update).

The paper benchmarks on the VLSI and TSP Art collections (Section 5.3), with a
top-N nearest-neighbour candidate graph per node (N=20 for VLSI, N=10 for Art).
Those datasets are not available here; these generators stand in for them:

* ``uniform_points``  -- n integer points uniform in [0, side]^2.
* ``mixture_points``  -- a fraction of the points from a mixture of isotropic
  clusters (the clustered density of TSP Art images), the rest uniform.
* ``knn_csr``         -- symmetrised k-nearest-neighbour candidate graph.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of a stream with key K is mix64(K + (i + 1) * golden_gamma).
Every operation below is integer or IEEE-754 basic arithmetic (+, -, *, / by
powers of two, floor), so the same seed gives the same points on every
platform; ``points_sha256`` fingerprints a point set.
"""
from __future__ import annotations

import hashlib

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags: each purpose draws from its own counter stream
TAG_UNIFORM = 1
TAG_CENTRE = 2
TAG_COMPONENT = 3
TAG_NORMAL = 4
TAG_BACKGROUND = 5


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (the published finaliser), elementwise on uint64."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: int) -> np.uint64:
    """Key of the counter stream for (seed, tag)."""
    base = np.array([(int(seed) * 0x100000001B3 + int(tag) * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                    dtype=np.uint64)
    return _mix64(base)[0]


def draws(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the stream with this key (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(key) + idx * _GAMMA)


def _bits_for(r: int) -> int:
    return max(1, int(r).bit_length())


def uniform_ints(key: np.uint64, count: int, hi: int, start: int = 0) -> tuple[np.ndarray, int]:
    """``count`` integers uniform in [0, hi] by rejection on the top bits.

    Returns (values int64, next unused draw index).  A draw v = x >> (64-b), with
    b the bit length of hi, is accepted when v <= hi; accepted draws keep stream
    order, so the result does not depend on how the stream is chunked.
    """
    b = _bits_for(hi)
    out = np.empty(count, dtype=np.int64)
    got = 0
    pos = start
    while got < count:
        need = count - got
        m = need + need // 8 + 64
        x = draws(key, pos, m) >> np.uint64(64 - b)
        ok = np.nonzero(x <= np.uint64(hi))[0]
        take = ok[:need]
        out[got:got + take.size] = x[take].astype(np.int64)
        got += take.size
        pos += int(take[-1]) + 1 if take.size == need else m
    return out, pos


def normal_deviates(key: np.uint64, index: np.ndarray) -> np.ndarray:
    """Approximately standard normal deviates, one per entry of ``index``.

    Irwin-Hall sum of twelve uniforms minus six (mean 0, variance 1, support
    [-6, 6]).  Deviate i uses draws 12*i .. 12*i+11; each uniform is the top 32
    bits of a draw, and the sum is formed exactly in integers before a single
    scaling by 2^-32, so the value is platform-independent.
    """
    index = np.asarray(index, dtype=np.uint64)
    acc = np.zeros(index.shape, dtype=np.int64)
    with np.errstate(over="ignore"):
        for j in range(12):
            ctr = index * np.uint64(12) + np.uint64(j + 1)
            x = _mix64(np.uint64(key) + ctr * _GAMMA) >> np.uint64(32)
            acc += x.astype(np.int64)
    return acc.astype(np.float64) * (2.0 ** -32) - 6.0


def uniform_points(n: int, seed: int, side: int = 1_000_000, tag: int = TAG_UNIFORM) -> np.ndarray:
    """n points with integer coordinates uniform in [0, side]^2, as int32 [n, 2]."""
    v, _ = uniform_ints(stream_key(seed, tag), 2 * n, side)
    return v.reshape(n, 2).astype(np.int32)


def mixture_points(n: int, seed: int, side: int = 1_000_000, frac: float = 0.7,
                   components: int = 100, sigma: float = 5000.0) -> np.ndarray:
    """round(frac*n) clustered points followed by n - round(frac*n) uniform points.

    Cluster centres are uniform in [0, side]^2; each clustered point picks its
    component uniformly, adds sigma times a normal deviate per axis and rounds
    to the nearest integer (floor(v + 0.5)).  A point that falls outside the box
    is redrawn with fresh deviates (same component) until it lands inside.
    """
    m = int(np.floor(frac * n + 0.5))
    cen, _ = uniform_ints(stream_key(seed, TAG_CENTRE), 2 * components, side)
    cen = cen.reshape(components, 2).astype(np.float64)
    comp, _ = uniform_ints(stream_key(seed, TAG_COMPONENT), m, components - 1)
    nkey = stream_key(seed, TAG_NORMAL)
    pts = np.empty((m, 2), dtype=np.int64)
    pending = np.arange(m, dtype=np.int64)
    attempt = 0
    while pending.size:
        base = (attempt * m + pending).astype(np.uint64) * np.uint64(2)
        gx = normal_deviates(nkey, base)
        gy = normal_deviates(nkey, base + np.uint64(1))
        px = np.floor(cen[comp[pending], 0] + sigma * gx + 0.5)
        py = np.floor(cen[comp[pending], 1] + sigma * gy + 0.5)
        inside = (px >= 0) & (px <= side) & (py >= 0) & (py <= side)
        sel = pending[inside]
        pts[sel, 0] = px[inside].astype(np.int64)
        pts[sel, 1] = py[inside].astype(np.int64)
        pending = pending[~inside]
        attempt += 1
    uni = uniform_points(n - m, seed, side, TAG_BACKGROUND).astype(np.int64) if n > m else np.zeros((0, 2), np.int64)
    return np.concatenate([pts, uni]).astype(np.int32)


def points_sha256(xy: np.ndarray) -> str:
    """SHA-256 of the little-endian int32 [n, 2] point array."""
    return hashlib.sha256(np.ascontiguousarray(xy, dtype="<i4").tobytes()).hexdigest()


def knn_csr(xy: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Symmetrised k-nearest-neighbour candidate graph as a CSR (row_ptr, col).

    The k nearest neighbours of u are the k other points with the smallest
    exact squared distance dx^2 + dy^2 (int64), ties broken by smaller index.
    Directed pairs u->w are then symmetrised (u~w if either lists the other),
    rows are sorted by column and hold no self-loop or duplicate.  A k-d tree
    proposes candidates; the exact order is decided on the int64 squared
    distances, and a row is re-queried with more candidates whenever the
    proposal could have cut a tie at the k-th place.
    """
    from scipy.spatial import cKDTree

    xy = np.asarray(xy, dtype=np.int64)
    n = xy.shape[0]
    if n < k + 1:
        raise ValueError("need n > k")
    tree = cKDTree(xy.astype(np.float64))
    nbr = np.empty((n, k), dtype=np.int64)
    rows = np.arange(n)
    kq = k + 9
    while rows.size:
        kk = min(kq, n)
        _, idx = tree.query(xy[rows].astype(np.float64), k=kk)
        idx = np.asarray(idx, dtype=np.int64).reshape(rows.size, kk)
        d = xy[idx] - xy[rows][:, None, :]
        d2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]
        key = d2 * n + idx
        key[idx == rows[:, None]] = np.iinfo(np.int64).max  # drop self
        order = np.argsort(key, axis=1, kind="stable")
        sk = np.take_along_axis(key, order, axis=1)
        sd2 = np.take_along_axis(d2, order, axis=1)
        sidx = np.take_along_axis(idx, order, axis=1)
        # the proposal is exact when the k-th kept distance is strictly below the
        # largest proposed distance (every point tied with it was then proposed)
        kth = sd2[:, k - 1]
        far = np.where(sk[:, -1] == np.iinfo(np.int64).max, sd2[:, -2], sd2[:, -1])
        exact = (kth < far) | (kk >= n)
        nbr[rows[exact]] = sidx[exact, :k]
        rows = rows[~exact]
        kq *= 2
    u = np.repeat(np.arange(n, dtype=np.int64), k)
    w = nbr.reshape(-1)
    keys = np.unique(np.concatenate([u * n + w, w * n + u]))
    src = keys // n
    col = (keys % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return row_ptr.astype(np.int32), col


def make_instance(kind: str, n: int, seed: int, k: int) -> dict:
    """Points plus candidate CSR for a named point distribution ('uniform' | 'mixture')."""
    if kind == "uniform":
        xy = uniform_points(n, seed)
    elif kind == "mixture":
        xy = mixture_points(n, seed)
    else:
        raise ValueError(kind)
    row_ptr, col = knn_csr(xy, k)
    return {"kind": kind, "n": n, "seed": seed, "k": k, "xy": xy,
            "row_ptr": row_ptr, "col": col, "sha256": points_sha256(xy)}


TAG_MLP_INIT = 6
TAG_FLOATS = 7


def uniform_floats(seed: int, count: int, lo: float, hi: float, tag: int = TAG_FLOATS) -> np.ndarray:
    """``count`` float32 values uniform in [lo, hi): the top 24 bits of each draw
    scaled by 2^-24 (exact in float32), then lo + (hi - lo) * u in float64."""
    u = (draws(stream_key(seed, tag), 0, count) >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
    return (lo + (hi - lo) * u).astype(np.float32)


# layout of the warm-start network's flat parameter vector (float32):
# W1 [128][16], b1 [128], W2 [128][128], b2 [128], w3 [128], b3 [1]
MLP_SIZES = (("W1", (128, 16)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
             ("w3", (128,)), ("b3", (1,)))
MLP_NPARAMS = sum(int(np.prod(s)) for _, s in MLP_SIZES)


def mlp_init(seed: int) -> np.ndarray:
    """Seeded initial parameters of the 16-128-128-1 network (float32 [18817]).

    Weights of a layer with fan-in m are uniform in [-sqrt(6/m), sqrt(6/m)) (He
    uniform, for ReLU); biases are zero except b3 = 0.5 (a neutral starting
    guess for lambda_v / s_v).
    """
    out = np.zeros(MLP_NPARAMS, dtype=np.float32)
    off = 0
    for i, (name, shape) in enumerate(MLP_SIZES):
        cnt = int(np.prod(shape))
        if name.startswith("W") or name == "w3":
            a = np.sqrt(6.0 / shape[-1]) if name != "w3" else np.sqrt(6.0 / 128)
            out[off:off + cnt] = uniform_floats(seed * 16 + i, cnt, -a, a, tag=TAG_MLP_INIT)
        elif name == "b3":
            out[off] = 0.5
        off += cnt
    return out
