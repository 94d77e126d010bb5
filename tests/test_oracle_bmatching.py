"""Pins of the oracle's degree-requirement generalisation (fractional b-matching).

Section 3 states the method for a general degree vector b (LP3): each node v
needs sum of x over delta(v) = b_v, and the GDP update uses the b_v-th and
(b_v+1)-th smallest adjusted edges.  These tests tie the b path to an
independent LP solver (HiGHS), to the assignment problem (b = 1 on a complete
bipartite graph, where the LP is integral), to brute force, to a complement
identity, to the coordinate-wise maximiser of the Lagrangian, and to the
b = 2 path itself.
"""
import numpy as np
import pytest

import instances as I
from test_oracle import complete_csr, edge_list, _isqrt_exact


def highs_opt_b(xy, row_ptr, col, b):
    """Fractional b-matching LP optimum on the CSR graph, by scipy's HiGHS."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    n = row_ptr.size - 1
    u, v, c = edge_list(xy, row_ptr, col)
    E = u.size
    A = coo_matrix((np.ones(2 * E), (np.concatenate([u, v]), np.concatenate([np.arange(E)] * 2))),
                   shape=(n, E)).tocsr()
    r = linprog(c.astype(float), A_eq=A, b_eq=np.asarray(b, dtype=float), bounds=(0, 1), method="highs")
    assert r.status == 0
    return r.fun


def lagrangian_row(t, zp, bv):
    """g(t) = b_v t + sum_e min(0, z'_e - t): the part of the Lagrangian that
    depends on lambda_v = t, with z'_e = c_e 2^F - lambda_u for the other end u."""
    return bv * t + np.minimum(0, zp - t).sum()


# ---- optimum value against independent solvers ------------------------------------

@pytest.mark.parametrize("n,seed", [(12, 0), (30, 1), (60, 2), (90, 3)])
def test_complete_graph_random_b_vs_highs(oracle_lib, n, seed):
    rng = np.random.default_rng(seed)
    xy = rng.integers(0, 10 ** 5, size=(n, 2)).astype(np.int32)
    b = rng.integers(1, 5, size=n).astype(np.int32)
    rp, col = complete_csr(n)
    r = oracle_lib.solve(xy, rp, col, b=b)
    assert r.status == 0 and r.certified == 2
    want = highs_opt_b(xy, rp, col, b)
    assert abs(r.opt - want) < 1e-6 * max(1.0, want)
    assert oracle_lib.certify(xy, r.row_ptr, r.col, r.x2, r.lam, r.frac_bits, r.bound2, b=b) == 0
    # the same point is not a fractional 2-matching unless b happens to be 2 everywhere
    assert oracle_lib.certify(xy, r.row_ptr, r.col, r.x2, r.lam, r.frac_bits, r.bound2) == 3


@pytest.mark.parametrize("kind,n,k,bmax", [("uniform", 400, 10, 3), ("mixture", 500, 12, 4)])
def test_candidate_graph_with_pricing_random_b_vs_complete_highs(oracle_lib, kind, n, k, bmax):
    inst = I.make_instance(kind, n, 8, k)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    b = np.random.default_rng(n).integers(1, bmax + 1, size=n).astype(np.int32)
    r = oracle_lib.solve(xy, rp, col, b=b)
    assert r.status == 0 and r.certified == 2
    krp, kcol = complete_csr(n)
    want = highs_opt_b(xy, krp, kcol, b)
    assert abs(r.opt - want) < 1e-6 * want


@pytest.mark.parametrize("m,seed", [(6, 0), (25, 1), (60, 2)])
def test_b1_complete_bipartite_is_the_assignment_problem(oracle_lib, m, seed):
    # K_{m,m} with b = 1: the LP is integral and its optimum is the assignment optimum
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(seed)
    xy = rng.integers(0, 10 ** 4, size=(2 * m, 2)).astype(np.int32)
    rows = [list(range(m, 2 * m))] * m + [list(range(m))] * m
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    d = xy[:m, None, :].astype(np.int64) - xy[None, m:, :]
    cmat = (_isqrt_exact(4 * (d[..., 0] ** 2 + d[..., 1] ** 2)) + 1) // 2
    ri, ci = linear_sum_assignment(cmat)
    r = oracle_lib.solve(xy, rp, col, b=1, pricing=False)
    assert r.status == 0 and r.certified >= 1
    assert r.opt == cmat[ri, ci].sum()


@pytest.mark.parametrize("n,seed", [(4, 0), (5, 1), (5, 2), (5, 3), (5, 4)])
def test_brute_force_tiny_random_b(oracle_lib, n, seed):
    rng = np.random.default_rng(seed)
    xy = rng.integers(0, 60, size=(n, 2)).astype(np.int32)
    b = rng.integers(1, n - 1, size=n).astype(np.int32)  # degree n - 1 >= b + 1
    rp, col = complete_csr(n)
    u, v, c = edge_list(xy, rp, col)
    # every half-integral x in {0, 1/2, 1}^E (Section 4), as x2 in {0, 1, 2}
    x2 = np.array(np.meshgrid(*([np.arange(3)] * u.size), indexing="ij")).reshape(u.size, -1).T
    inc = np.zeros((u.size, n), dtype=np.int64)
    inc[np.arange(u.size), u] = 1
    inc[np.arange(u.size), v] = 1
    ok = np.all(x2 @ inc == 2 * b, axis=1)
    r = oracle_lib.solve(xy, rp, col, b=b)
    if not ok.any():
        assert r.status != 0
    else:
        assert r.status == 0 and r.opt == (x2[ok] @ c).min() / 2.0


def test_complement_identity(oracle_lib):
    # On K_n, x is a fractional (n-2)-matching exactly when y = 1 - x is a
    # fractional perfect matching, so opt(b = n-2) = total edge cost minus the
    # MAXIMUM cost of a fractional perfect matching (HiGHS on the negated costs).
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    n = 40
    rng = np.random.default_rng(11)
    xy = rng.integers(0, 5000, size=(n, 2)).astype(np.int32)
    rp, col = complete_csr(n)
    u, v, c = edge_list(xy, rp, col)
    E = u.size
    A = coo_matrix((np.ones(2 * E), (np.concatenate([u, v]), np.concatenate([np.arange(E)] * 2))),
                   shape=(n, E)).tocsr()
    ymax = -linprog(-c.astype(float), A_eq=A, b_eq=np.ones(n), bounds=(0, 1), method="highs").fun
    rn = oracle_lib.solve(xy, rp, col, b=n - 2)
    assert rn.status == 0 and rn.certified == 2
    assert abs(rn.opt - (c.sum() - ymax)) < 1e-6 * rn.opt


# ---- the GDP sweep with general b ---------------------------------------------------

@pytest.mark.parametrize("bval", [1, 3, 5])
def test_full_step_lands_on_the_coordinate_maximiser(oracle_lib, bval):
    # shift = 1 (no damping): each new lambda_v must maximise g over lambda_v with
    # the other duals fixed (the coordinate ascent step of Section 3).  Checked
    # against g evaluated at every breakpoint, with no order statistic involved.
    inst = I.make_instance("uniform", 300, 4, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    rng = np.random.default_rng(bval)
    lam = rng.integers(0, 3000 * 256, size=300).astype(np.int32)
    b = np.where(rng.random(300) < 0.5, bval, 2).astype(np.int32)
    st, new, _, _ = oracle_lib.sweep(rp, col, cost, lam, 8, 1, b=b)
    assert st == 0
    for v in range(300):
        e = slice(rp[v], rp[v + 1])
        zp = (cost[e].astype(np.int64) << 8) - lam[col[e]]
        best = max(lagrangian_row(t, zp, b[v]) for t in zp)
        assert lagrangian_row(int(new[v]), zp, b[v]) == best


def test_b2_everywhere_equals_default(oracle_lib):
    inst = I.make_instance("mixture", 600, 3, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    a = oracle_lib.gdp(rp, col, cost, np.zeros(600, np.int32), 8, 2, 3000, trace=True)
    c = oracle_lib.gdp(rp, col, cost, np.zeros(600, np.int32), 8, 2, 3000, trace=True, b=2)
    assert a[0] == c[0] and a[2] == c[2]
    assert np.array_equal(a[1], c[1]) and np.array_equal(a[3], c[3])
    r0 = oracle_lib.solve(xy, rp, col)
    r2 = oracle_lib.solve(xy, rp, col, b=np.full(600, 2, np.int32))
    assert r0.bound2 == r2.bound2 and np.array_equal(r0.lam, r2.lam) and np.array_equal(r0.x2, r2.x2)


def test_bound_below_opt_every_sweep_random_b(oracle_lib):
    # weak duality: every sweep's bound is at most the LP optimum
    inst = I.make_instance("uniform", 200, 6, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    b = np.random.default_rng(2).integers(1, 5, size=200).astype(np.int32)
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam, it, tb, _ = oracle_lib.gdp(rp, col, cost, np.zeros(200, np.int32), 8, 2, 20000,
                                        trace=True, b=b)
    opt = highs_opt_b(xy, rp, col, b)
    assert it > 10 and np.all(tb / 512.0 <= opt + 1e-9)
    assert tb[-1] / 512.0 > 0.97 * opt


def test_degree_below_b_plus_one_is_invalid(oracle_lib):
    inst = I.make_instance("uniform", 100, 1, 4)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    b = np.full(100, 2, np.int32)
    b[17] = int(rp[18] - rp[17])  # needs degree b + 1
    st, *_ = oracle_lib.sweep(rp, col, cost, np.zeros(100, np.int32), 8, 2, b=b)
    assert st == oracle_lib.OR_INVALID
    b[17] = 0
    st, *_ = oracle_lib.sweep(rp, col, cost, np.zeros(100, np.int32), 8, 2, b=b)
    assert st == oracle_lib.OR_INVALID
