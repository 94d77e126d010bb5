"""The full pricing scan on the tensor cores (F2M_FLAG_PRICING_TENSOR) against
the CPU oracle and against the default fp32 scan, through the C ABI.

The tensor-core filter quantises the points of a tile pair to 10-bit integers
in a frame fitted to the pair and decides |D|^2 < (R_u + R_v)^2 from one fp16
matrix product with an fp32 accumulator; its no-false-negative argument needs
that accumulator to be exact for the operand ranges it produces, which
f2m_pricing_mma_check tests directly.  The scans are compared pair set by pair
set with the oracle's plain double loop (exact integers) on inputs that push
the frame: coordinates at both ends of [0, 2^20), coincident points, a dense
cluster next to far points, lambdas near +-2^29 and negative ones, and sizes
that leave ragged 128-point tiles; whole solves and a batch agree with the
default scan bit for bit.
"""
import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from paper_2011_08170_gb300 import build as B

pytestmark = pytest.mark.gpu

TENSOR = f2m.F2M_FLAG_PRICING_TENSOR


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def _sorted(p):
    p = np.asarray(p).reshape(-1, 2)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def _scan(xy, rp, col, lam, fb, flags=0):
    ctx = f2m.f2m_create(xy, rp, col, f2m.f2m_default_params(flags=flags))
    f2m.f2m_set_lambda(ctx, lam, fb)
    cnt, pairs = f2m.f2m_price(ctx)
    return cnt, _sorted(pairs)


def _check(O, xy, lam, fb, k=4):
    rp, col = O.knn_csr(xy, k)
    cnt_o, pairs_o = O.pricing(xy, rp, col, lam, fb)
    cnt, pairs = _scan(xy, rp, col, lam, fb, TENSOR)
    assert cnt == cnt_o
    assert np.array_equal(pairs, pairs_o)
    cnt2, pairs2 = _scan(xy, rp, col, lam, fb)
    assert cnt2 == cnt_o and np.array_equal(pairs2, pairs_o)
    return cnt


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_tensor_core_accumulator_is_exact(lib, seed):
    checked, bad = f2m.f2m_pricing_mma_check(48, seed)
    assert checked == 48 * 128 * 128
    assert bad == 0


@pytest.mark.parametrize("n", [8, 127, 128, 129, 255, 256, 257, 383, 385, 1000])
def test_ragged_sizes(lib, O, n):
    d = I.make_instance("uniform", n, 40 + n, 4) if n >= 8 else None
    rng = np.random.default_rng(n)
    xy = d["xy"] if d is not None else rng.integers(0, 1 << 20, size=(n, 2)).astype(np.int32)
    fb = 8
    lam = (rng.integers(0, 120000, size=n) << fb).astype(np.int32)
    _check(O, xy, lam, fb, k=min(4, n - 1))


def test_coordinates_at_both_ends(lib, O):
    # corners of [0, 2^20) and points on the edges: the frame spans the whole
    # range (shift 10) and the quantised coordinates reach 0 and 1023
    rng = np.random.default_rng(7)
    m = (1 << 20) - 1
    corners = np.array([[0, 0], [m, m], [0, m], [m, 0], [1, 1], [m - 1, m - 1]], np.int64)
    edge = rng.integers(0, 1 << 20, size=(600, 2))
    edge[:300, 0] = rng.choice([0, m], size=300)
    edge[300:, 1] = rng.choice([0, m], size=300)
    xy = np.concatenate([corners, edge]).astype(np.int32)
    n = xy.shape[0]
    lam = (rng.integers(0, 700000, size=n) << 8).astype(np.int32)
    assert _check(O, xy, lam, 8) > 0


def test_coincident_points_and_a_dense_cluster(lib, O):
    # groups of identical points (distance 0, cost 0), a cluster 40 units
    # wide, and far points around it: tile pairs with a box of extent 0, tiny
    # ones, and ones that mix the cluster with far points
    rng = np.random.default_rng(8)
    dup = np.repeat(rng.integers(0, 1 << 20, size=(40, 2)), 5, axis=0)
    cl = 500000 + rng.integers(0, 40, size=(700, 2))
    far = rng.integers(0, 1 << 20, size=(500, 2))
    xy = np.concatenate([dup, cl, far]).astype(np.int32)
    n = xy.shape[0]
    lam = rng.integers(-2000, 30000, size=n).astype(np.int32)
    lam[:200] = rng.integers(1, 50, size=200)  # coincident points: any lam_u + lam_v > 0 prices
    assert _check(O, xy, lam, 8) > 0


def test_extreme_lambdas(lib, O):
    # lambdas near +-2^29 (radii that force the coarsest frames), very negative
    # ones (radius 0) and zeros, at both fractional precisions
    rng = np.random.default_rng(9)
    n = 900
    d = I.make_instance("mixture", n, 9, 5)
    for fb in (8, 9):
        lam = rng.integers(-50000, 400000, size=n).astype(np.int64)
        lam[:6] = (1 << 29) - 1 - rng.integers(0, 1000, size=6)
        lam[6:40] = -(1 << 29) + 1 + rng.integers(0, 1000, size=34)
        lam[40:60] = 0
        _check(O, d["xy"], lam.astype(np.int32), fb)


@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 20000, 3, 10), ("mixture", 30000, 4, 12)])
def test_tensor_core_scan_equals_fp32_scan(lib, O, kind, n, seed, k):
    # a converged-like lambda (GDP from 0) plus noise: many pairs near the
    # boundary, the same pair set from both filters and from the oracle
    d = I.make_instance(kind, n, seed, k)
    rp, col = d["row_ptr"], d["col"]
    cost = O.cost_table(d["xy"], rp, col)
    _, lam, *_ = O.gdp(rp, col, cost, np.zeros(n, np.int32), 8, 2, 64)
    rng = np.random.default_rng(seed)
    lam = (lam + rng.integers(0, 600, size=n)).astype(np.int32)
    cnt_o, pairs_o = O.pricing(d["xy"], rp, col, lam, 8)
    cnt, pairs = _scan(d["xy"], rp, col, lam, 8, TENSOR)
    cnt2, pairs2 = _scan(d["xy"], rp, col, lam, 8)
    assert cnt == cnt2 == cnt_o > 0
    assert np.array_equal(pairs, pairs_o) and np.array_equal(pairs2, pairs_o)


def test_whole_solves_with_the_tensor_core_scan(lib, O):
    # the scan's pair sets are those of the default scan, so whole solves agree
    # bit for bit: counters, optimum, lambda, x and the candidate graph; and a
    # batch (several segments, each scanned on its own) agrees with its default
    for kind, n, seed, k in (("uniform", 6000, 1, 4), ("mixture", 9000, 2, 6)):
        d = I.make_instance(kind, n, seed, k)
        a = f2m.solve(d["xy"], d["row_ptr"], d["col"])
        b = f2m.solve(d["xy"], d["row_ptr"], d["col"], params=f2m.f2m_default_params(flags=TENSOR))
        for key in ("status", "iterations", "phases", "pricing_rounds", "edges_added", "finisher_calls",
                    "augmentations", "bound2", "frac_bits", "certified"):
            assert a.info[key] == b.info[key], key
        assert a.info["edges_added"] > 0
        assert np.array_equal(a.lam, b.lam) and np.array_equal(a.x2, b.x2) and np.array_equal(a.col, b.col)
    ds = [I.make_instance("uniform" if i % 2 else "mixture", 700 + 300 * i, 60 + i, 5) for i in range(6)]
    insts = [(d["xy"], d["row_ptr"], d["col"]) for d in ds]
    out = []
    for fl in (0, TENSOR):
        bt = f2m.f2m_create_batch(insts, f2m.f2m_default_params(flags=fl))
        infos, tot = f2m.f2m_solve_batch(bt)
        assert tot.status == 0 and tot.certified == 2
        out.append([(i.iterations, i.pricing_rounds, i.edges_added, i.bound2, *f2m.f2m_batch_get_lambda(bt, s))
                    for s, i in enumerate(infos)])
    for x, y in zip(*out):
        assert x[:4] == y[:4] and np.array_equal(x[4], y[4]) and x[5] == y[5]
