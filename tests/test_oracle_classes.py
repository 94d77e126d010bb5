"""Pins of the oracle's class-by-class (Gauss-Seidel) sweep and its colouring.

The variant updates one colour class (an independent set) at a time from the
current lambda.  With the full step each class update is exact block
coordinate ascent on the Lagrangian, so the bound cannot fall; these tests tie
it to that fact, to the coordinate maximiser of the Lagrangian, to relabelling
invariance, to HiGHS through the whole solve, and the hash behind the colouring
to SplitMix64's published output.
"""
import numpy as np
import pytest

import instances as I
from test_oracle import complete_csr, highs_opt
from test_oracle_bmatching import highs_opt_b, lagrangian_row


def test_splitmix64_published_sequence(oracle_lib):
    # SplitMix64 from state 0 yields e220a8397b1dcdaf, 6e789e6aa1b965f4,
    # 06c45d188009454f, ...; output k is the first output seeded with k * gamma
    gamma = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for k, w in enumerate(want):
        assert oracle_lib.splitmix64((k * gamma) % (1 << 64)) == w


@pytest.mark.parametrize("kind,n,k", [("uniform", 2000, 10), ("mixture", 3000, 6), ("uniform", 500, 16)])
def test_colouring_is_proper_and_greedy(oracle_lib, kind, n, k):
    d = I.make_instance(kind, n, 2, k)
    rp, col = d["row_ptr"], d["col"]
    nc, color = oracle_lib.color_greedy(rp, col)
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(color[src] != color[col])            # proper
    assert nc == color.max() + 1 and nc <= np.diff(rp).max() + 1
    for v in range(n):                                 # every smaller colour is blocked
        nb = set(color[col[rp[v]:rp[v + 1]]].tolist())
        assert all(c in nb for c in range(color[v]))


def test_colouring_special_graphs(oracle_lib):
    # K_n: all degrees equal, so the colours rank the nodes by the hash, largest first
    n = 30
    rp, col = complete_csr(n)
    nc, color = oracle_lib.color_greedy(rp, col)
    h = np.array([oracle_lib.splitmix64(v) for v in range(n)], dtype=np.uint64)
    assert nc == n and np.array_equal(np.argsort(color), np.argsort(-h.astype(np.float64), kind="stable"))
    # complete bipartite K_{m,m}: any greedy order gives two colours, one per side
    m = 12
    rows = [list(range(m, 2 * m))] * m + [list(range(m))] * m
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    nc, color = oracle_lib.color_greedy(rp, col)
    assert nc == 2 and len(set(color[:m])) == 1 and len(set(color[m:])) == 1


def test_full_step_bound_never_decreases(oracle_lib):
    d = I.make_instance("uniform", 1500, 3, 10)
    rp, col = d["row_ptr"], d["col"]
    cost = oracle_lib.cost_table(d["xy"], rp, col)
    nc, color = oracle_lib.color_greedy(rp, col)
    st, lam, it, tb, tc = oracle_lib.gdp_gs(rp, col, cost, np.zeros(1500, np.int32), color, nc,
                                            8, 1, 50000, trace=True)
    assert st == oracle_lib.OR_OK and it > 20
    assert np.all(np.diff(tb) >= 0)
    # the bound at the fixed point is below the LP optimum on this graph
    assert oracle_lib.bound2(rp, col, cost, lam, 8) / 512.0 <= highs_opt(d["xy"], rp, col) + 1e-9


@pytest.mark.parametrize("bval", [None, 3])
def test_each_class_lands_on_the_coordinate_maximiser(oracle_lib, bval):
    # replay the sweep one class at a time: nodes of colour >= c are parked in a
    # colour that the sweep never reaches
    d = I.make_instance("mixture", 600, 4, 10)
    rp, col = d["row_ptr"], d["col"]
    cost = oracle_lib.cost_table(d["xy"], rp, col)
    nc, color = oracle_lib.color_greedy(rp, col)
    b = None if bval is None else np.where(np.arange(600) % 3 == 0, bval, 2).astype(np.int32)
    bv = np.full(600, 2) if b is None else b
    lam0 = np.random.default_rng(1).integers(0, 4000 * 256, size=600).astype(np.int32)
    _, full, _, _ = oracle_lib.gs_sweep(rp, col, cost, lam0, color, nc, 8, 1, b=b)
    for c in range(nc):
        part = np.where(color < c, color, nc).astype(np.int32)
        _, before, _, _ = oracle_lib.gs_sweep(rp, col, cost, lam0, part, nc, 8, 1, b=b)
        part = np.where(color <= c, color, nc).astype(np.int32)
        _, after, _, _ = oracle_lib.gs_sweep(rp, col, cost, lam0, part, nc, 8, 1, b=b)
        for v in np.nonzero(color == c)[0]:
            zp = (cost[rp[v]:rp[v + 1]].astype(np.int64) << 8) - before[col[rp[v]:rp[v + 1]]]
            best = max(lagrangian_row(t, zp, bv[v]) for t in zp)
            assert lagrangian_row(int(after[v]), zp, bv[v]) == best
        assert np.array_equal(after[color > c], lam0[color > c])
    assert np.array_equal(after, full)


def test_relabelling_invariance(oracle_lib):
    d = I.make_instance("uniform", 800, 5, 8)
    rp, col, xy = d["row_ptr"], d["col"], d["xy"]
    cost = oracle_lib.cost_table(xy, rp, col)
    nc, color = oracle_lib.color_greedy(rp, col)
    st, lam, it, tb, _ = oracle_lib.gdp_gs(rp, col, cost, np.zeros(800, np.int32), color, nc,
                                           8, 2, 20000, trace=True)
    perm = np.random.default_rng(9).permutation(800)  # new node i is old node perm[i]
    inv = np.argsort(perm)
    pxy = xy[perm]
    prp, pcol = I.knn_csr(pxy, 8)
    pcost = oracle_lib.cost_table(pxy, prp, pcol)
    st2, lam2, it2, tb2, _ = oracle_lib.gdp_gs(prp, pcol, pcost, np.zeros(800, np.int32),
                                               color[perm], nc, 8, 2, 20000, trace=True)
    assert st == st2 and it == it2 and np.array_equal(tb, tb2)
    assert np.array_equal(lam2, lam[perm]) and np.array_equal(lam2[inv], lam)


@pytest.mark.parametrize("kind,n,k,b", [("uniform", 400, 10, None), ("mixture", 500, 8, None),
                                        ("uniform", 300, 10, 3)])
def test_class_solve_reaches_the_lp_optimum(oracle_lib, kind, n, k, b):
    d = I.make_instance(kind, n, 6, k)
    xy, rp, col = d["xy"], d["row_ptr"], d["col"]
    for shift in (1, 2):
        r = oracle_lib.solve(xy, rp, col, classes=True, shift=shift, b=b)
        assert r.status == 0 and r.certified == 2
        krp, kcol = complete_csr(n)
        want = highs_opt(xy, krp, kcol) if b is None else highs_opt_b(xy, krp, kcol, np.full(n, b))
        assert abs(r.opt - want) < 1e-6 * want
        assert oracle_lib.certify(xy, r.row_ptr, r.col, r.x2, r.lam, r.frac_bits, r.bound2, b=b) == 0


def test_class_sweep_overflow_keeps_value(oracle_lib):
    # a huge lambda pushes a node past 2^29: it keeps its value, the sweep completes
    d = I.make_instance("uniform", 200, 1, 6)
    rp, col = d["row_ptr"], d["col"]
    cost = oracle_lib.cost_table(d["xy"], rp, col)
    nc, color = oracle_lib.color_greedy(rp, col)
    lam = np.zeros(200, np.int32)
    v = int(np.argmax(color == 0))
    lam[col[rp[v]:rp[v + 1]]] = -(1 << 29) + 64  # neighbours far below: z near 2^29 for v
    st, out, _, ch = oracle_lib.gs_sweep(rp, col, cost, lam, color, nc, 8, 1)
    assert st == oracle_lib.OR_OVERFLOW and out[v] == 0 and ch > 0
