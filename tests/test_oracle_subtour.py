"""Pins of the oracle's GDP with subtour-elimination cuts (oracle/subtour.c).

The LP is Section 4's F2M plus cuts x(delta(S)) >= 2 (the relaxation the
paper's Discussion names next), all constraints of Section 3's class (8).
Each part is pinned to something other than the oracle itself: connected
components against scipy, the Lagrangian bound against HiGHS (weak duality at
every sweep, and equality at HiGHS's own optimal duals), each cut update
against the exact maximiser of its part of the Lagrangian, the cut-free sweep
against the plain F2M sweep, pricing against a numpy all-pairs scan.
"""
import numpy as np
import pytest

import instances as I


def _edges(rp, col):
    n = rp.size - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    m = src < col
    return src[m], col[m]


def highs_cut_lp(rp, col, cost, cuts):
    """The cut LP on the candidate graph by HiGHS: (optimum, lam*, mu*)."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    n = rp.size - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    m = src < col
    u, v, c = src[m], col[m], cost[m].astype(float)
    E = u.size
    A = coo_matrix((np.ones(2 * E), (np.concatenate([u, v]), np.concatenate([np.arange(E)] * 2))),
                   shape=(n, E)).tocsr()
    rows, cols, k = [], [], 0
    for l in range(cuts.L):
        cl = cuts.comp[l]
        for s in range(cuts.ncuts[l]):
            cr = np.nonzero((cl[u] == s) != (cl[v] == s))[0]
            rows += [k] * cr.size
            cols += cr.tolist()
            k += 1
    G = coo_matrix((-np.ones(len(rows)), (rows, cols)), shape=(k, E)).tocsr()
    r = linprog(c, A_ub=G, b_ub=-2 * np.ones(k), A_eq=A, b_eq=2 * np.ones(n), bounds=(0, 1),
                method="highs")
    assert r.status == 0
    return r.fun, r.eqlin.marginals, -r.ineqlin.marginals


def f2m_with_cuts(O, kind, n, seed, k):
    d = I.make_instance(kind, n, seed, k)
    xy, rp, col = d["xy"], d["row_ptr"], d["col"]
    cost = O.cost_table(xy, rp, col)
    r = O.solve(xy, rp, col, pricing=False)  # the F2M optimum on the candidate graph
    comp, m = O.separate(r.row_ptr, r.col, r.x2)
    return d, cost, r, O.Cuts(n, [(comp, m)])


def test_separation_equals_scipy_components(oracle_lib):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    O = oracle_lib
    for kind, n, seed in (("uniform", 400, 1), ("mixture", 600, 2)):
        d = I.make_instance(kind, n, seed, 8)
        xy, rp, col = d["xy"], d["row_ptr"], d["col"]
        r = O.solve(xy, rp, col, pricing=False)
        comp, m = O.separate(r.row_ptr, r.col, r.x2)
        src = np.repeat(np.arange(n), np.diff(r.row_ptr))
        keep = r.x2 > 0
        g = coo_matrix((np.ones(keep.sum()), (src[keep], r.col[keep])), shape=(n, n))
        nc, lab = connected_components(g, directed=False)
        assert nc >= 3
        # components numbered by their smallest node
        first = np.full(nc, n)
        np.minimum.at(first, lab, np.arange(n))
        order = np.argsort(first)
        rank = np.empty(nc, int)
        rank[order] = np.arange(nc)
        want = rank[lab]
        # a component is a cut unless fewer than 3 candidate edges cross it
        s2 = np.repeat(np.arange(n), np.diff(rp))
        cross = np.bincount(want[s2][want[s2] != want[col]], minlength=nc)
        ids = np.cumsum(cross >= 3) - 1
        exp = np.where(cross[want] >= 3, ids[want], -1)
        assert m == int((cross >= 3).sum()) and np.array_equal(comp, exp)


def test_two_components_give_one_cut_without_node_0(oracle_lib):
    # two far-apart squares: the support has two components, delta(S) is the
    # same set for S and its complement, so one cut -- the square without node 0
    xy = np.array([[0, 0], [0, 10], [10, 10], [10, 0], [1000, 0], [1000, 10], [1010, 10], [1010, 0]],
                  dtype=np.int32)
    rp = np.arange(0, 8 * 7 + 1, 7, dtype=np.int32)
    col = np.array([j for i in range(8) for j in range(8) if j != i], dtype=np.int32)
    r = oracle_lib.solve(xy, rp, col, pricing=False)
    comp, m = oracle_lib.separate(r.row_ptr, r.col, r.x2)
    assert m == 1 and list(comp) == [-1] * 4 + [0] * 4


def test_no_cuts_equals_plain_sweep(oracle_lib):
    O = oracle_lib
    d = I.make_instance("mixture", 800, 3, 10)
    xy, rp, col = d["xy"], d["row_ptr"], d["col"]
    cost = O.cost_table(xy, rp, col)
    rng = np.random.default_rng(0)
    lam = rng.integers(-(1 << 22), 1 << 22, size=800).astype(np.int32)
    empty = O.Cuts(800)
    for shift in (1, 2):
        st, nl, nm, b2, ch = O.cut_sweep(rp, col, cost, empty, lam, None, 8, shift)
        st0, nl0, b20, ch0 = O.sweep(rp, col, cost, lam, 8, shift)
        assert st == st0 and np.array_equal(nl, nl0) and b2 == b20 and ch == ch0


@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 300, 0, 10), ("mixture", 250, 5, 8)])
def test_bound_below_cut_lp_optimum_every_sweep_and_close_to_it(oracle_lib, kind, n, seed, k):
    O = oracle_lib
    d, cost, r, cuts = f2m_with_cuts(O, kind, n, seed, k)
    opt, _, _ = highs_cut_lp(d["row_ptr"], d["col"], cost, cuts)
    assert cuts.total >= 3 and opt > r.opt  # the cuts bind
    st, lam, mu, it, tb, tc = O.cut_gdp(d["row_ptr"], d["col"], cost, cuts, r.lam >> 1, None, 8, 2, 6000,
                                        trace=True)
    assert st in (O.OR_OK, O.OR_NOT_CONVERGED) and np.all(mu >= 0)
    assert np.all(tb / 512.0 <= opt + 1e-6)                 # weak duality, every sweep
    assert tb.max() / 512.0 >= opt - 5e-3 * opt             # within 0.5% of the cut LP optimum
    assert tb.max() / 512.0 > r.opt                         # above the F2M optimum


def test_bound_formula_at_highs_duals(oracle_lib):
    # strong duality: at the LP's optimal duals the Lagrangian bound equals the
    # optimum.  The duals are rounded to the 2^-8 grid; each rounding moves the
    # bound by at most half a unit times the constraint's size plus 2.
    O = oracle_lib
    d, cost, r, cuts = f2m_with_cuts(O, "uniform", 200, 4, 10)
    rp, col = d["row_ptr"], d["col"]
    opt, lam_f, mu_f = highs_cut_lp(rp, col, cost, cuts)
    lam = np.rint(lam_f * 256).astype(np.int32)
    mu = np.rint(np.maximum(mu_f, 0) * 256).astype(np.int32)
    b = O.cut_bound2(rp, col, cost, cuts, lam, mu, 8) / 512.0
    deg = np.diff(rp)
    u, v = _edges(rp, col)
    cross = [int(((cuts.comp[0][u] == s) != (cuts.comp[0][v] == s)).sum()) for s in range(cuts.total)]
    slack = (0.5 / 256) * (float((deg + 2).sum()) + float(sum(c + 2 for c in cross)))
    assert abs(b - opt) <= slack, (b, opt, slack)
    # and a planted mistake in the formula (cut duals left out of z) is far off
    b_wrong = O.bound2(rp, col, cost, lam, 8) / 512.0 + 2 * mu.sum() / 256.0
    assert abs(b_wrong - opt) > 10 * slack


def _cut_part(zp, mu):
    """2 mu + sum over the cut's edges of min(0, z' - mu) (z' = z without this mu)."""
    return 2 * mu + np.minimum(0, zp - mu).sum()


def test_cut_step_moves_toward_the_maximiser_of_its_part_of_the_lagrangian(oracle_lib):
    # Section 3's gradient for a cut: its part of the Lagrangian, as a function
    # of mu_S >= 0 with every other dual at the sweep's input, is concave and
    # piecewise linear with its maxima between the 2nd and 3rd smallest z'
    # (z without mu_S).  A sweep's mu_S must never lower it (the damped step
    # moves toward the maximisers, never past them), and a mu_S already among
    # the maximisers stays there.  A wrong order statistic fails both.
    O = oracle_lib
    d, cost, r, cuts = f2m_with_cuts(O, "mixture", 300, 6, 10)
    rp, col, xy = d["row_ptr"], d["col"], d["xy"]
    rng = np.random.default_rng(1)
    lam = (r.lam >> 1) + rng.integers(-3000, 3000, size=300).astype(np.int32)
    u, v = _edges(rp, col)
    cl = cuts.comp[0]
    # odd cuts: random duals; even cuts: a point among their maximisers given
    # the duals set so far (a neighbouring even cut set later can move it out)
    mu = np.where(np.arange(cuts.total) % 2 == 1, rng.integers(0, 200000, size=cuts.total), 0).astype(np.int32)
    for s in range(0, cuts.total, 2):
        cr = np.nonzero((cl[u] == s) != (cl[v] == s))[0]
        zs = np.sort([O.cut_z(xy, cuts, lam, mu, 8, int(u[e]), int(v[e])) for e in cr])
        lo, hi = max(0, int(zs[1])), int(zs[2])
        if hi >= lo:
            mu[s] = rng.integers(lo, hi + 1)
    zp_all = []
    for s in range(cuts.total):
        cr = np.nonzero((cl[u] == s) != (cl[v] == s))[0]
        zp_all.append(np.array([O.cut_z(xy, cuts, lam, mu, 8, int(u[e]), int(v[e])) for e in cr]) + mu[s])
    inside = 0
    for shift in (1, 2):
        st, nl, nm, b2, ch = O.cut_sweep(rp, col, cost, cuts, lam, mu, 8, shift)
        for s in range(cuts.total):
            zp = zp_all[s]
            best = max(_cut_part(zp, m) for m in [0] + [int(t) for t in zp if t >= 0])
            assert _cut_part(zp, nm[s]) >= _cut_part(zp, mu[s]), (shift, s)
            if _cut_part(zp, mu[s]) == best:
                inside += 1
                assert _cut_part(zp, nm[s]) == best, (shift, s)
    assert inside >= cuts.total // 4


def test_cut_pricing_equals_numpy_scan(oracle_lib):
    O = oracle_lib
    d, cost, r, cuts = f2m_with_cuts(O, "uniform", 350, 7, 5)
    xy, rp, col = d["xy"], d["row_ptr"], d["col"]
    rng = np.random.default_rng(2)
    lam = (r.lam >> 1) + rng.integers(0, 20000, size=350).astype(np.int32)
    mu = rng.integers(0, 60000, size=cuts.total).astype(np.int32)
    cnt, pairs = O.cut_pricing(xy, rp, col, cuts, lam, mu, 8)
    iu, iv = np.triu_indices(350, 1)
    dd = xy[iu].astype(np.int64) - xy[iv]
    d2 = dd[:, 0] ** 2 + dd[:, 1] ** 2
    c = np.floor(np.sqrt(d2) + 0.5).astype(np.int64)
    cu, cv = cuts.comp[0][iu], cuts.comp[0][iv]
    term = np.where(cu != cv, np.where(cu >= 0, mu[np.maximum(cu, 0)], 0) +
                    np.where(cv >= 0, mu[np.maximum(cv, 0)], 0), 0)
    neg = (c << 8) - lam[iu].astype(np.int64) - lam[iv] - term < 0
    src = np.repeat(np.arange(350), np.diff(rp))
    incsr = set(zip(src.tolist(), col.tolist()))
    want = [(a, b) for a, b in zip(iu[neg].tolist(), iv[neg].tolist()) if (a, b) not in incsr]
    assert cnt == len(want) > 0 and [tuple(p) for p in pairs.tolist()] == want


def test_cut_overflow_and_short_cut(oracle_lib):
    O = oracle_lib
    d, cost, r, cuts = f2m_with_cuts(O, "uniform", 300, 0, 10)
    rp, col = d["row_ptr"], d["col"]
    # every lambda at -2^28: each crossing z is c 2^8 + 2^29 - mu, so a cut
    # dual just below 2^29 is pushed up past it
    lam = np.full(300, -(1 << 28), np.int32)
    mu = np.zeros(cuts.total, np.int32)
    mu[0] = (1 << 29) - 2
    st, nl, nm, b2, _ = O.cut_sweep(rp, col, cost, cuts, lam, mu, 8, 2)
    assert st == O.OR_OVERFLOW and nm[0] >= 0
    # the bound of the overflowing sweep is still the whole bound at its input
    assert b2 == O.cut_bound2(rp, col, cost, cuts, lam, mu, 8)
    # two K_4 joined by two edges: the cut around one K_4 has 2 crossing
    # edges, fewer than the 3 values Section 3's gradient takes -> refused
    xy = np.array([[0, 0], [0, 9], [9, 0], [9, 9], [50, 0], [50, 9], [59, 0], [59, 9]], np.int32)
    nb = [[1, 2, 3, 4], [0, 2, 3, 5], [0, 1, 3], [0, 1, 2], [0, 5, 6, 7], [1, 4, 6, 7], [4, 5, 7], [4, 5, 6]]
    rp2 = np.concatenate([[0], np.cumsum([len(x) for x in nb])]).astype(np.int32)
    col2 = np.array([c for x in nb for c in sorted(x)], np.int32)
    c2 = O.cost_table(xy, rp2, col2)
    short = O.Cuts(8, [(np.array([0, 0, 0, 0, -1, -1, -1, -1], np.int32), 1)])
    st, *_ = O.cut_sweep(rp2, col2, c2, short, np.zeros(8, np.int32), None, 8, 2)
    assert st == O.OR_INVALID
