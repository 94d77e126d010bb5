"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test ties one part of the oracle to the paper or to mathematics:
hand-worked values (tests/golden), closed forms, brute force on tiny inputs,
an independent LP solver (HiGHS via scipy), weak duality, and invariants.
"""
import json
import math
import os

import numpy as np
import pytest

import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _isqrt_exact(a: np.ndarray) -> np.ndarray:
    """floor(sqrt(a)) for int64 a, corrected in integers."""
    r = np.floor(np.sqrt(a.astype(np.float64))).astype(np.int64)
    r = np.where(r * r > a, r - 1, r)
    r = np.where((r + 1) * (r + 1) <= a, r + 1, r)
    return r


def complete_csr(n):
    row_ptr = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int32)
    col = np.array([j for i in range(n) for j in range(n) if j != i], dtype=np.int32)
    return row_ptr, col


def edge_list(xy, row_ptr, col):
    n = row_ptr.size - 1
    src = np.repeat(np.arange(n), np.diff(row_ptr))
    m = src < col
    u, v = src[m], col[m].astype(np.int64)
    d = xy[u].astype(np.int64) - xy[v].astype(np.int64)
    d2 = d[:, 0] ** 2 + d[:, 1] ** 2
    c = (_isqrt_exact(4 * d2) + 1) // 2  # nearest integer to sqrt(d2), integer-exact
    return u, v, c


def highs_opt(xy, row_ptr, col):
    """F2M LP optimum (Section 4) on the CSR graph, by scipy's HiGHS."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    n = row_ptr.size - 1
    u, v, c = edge_list(xy, row_ptr, col)
    E = u.size
    A = coo_matrix((np.ones(2 * E), (np.concatenate([u, v]), np.concatenate([np.arange(E)] * 2))),
                   shape=(n, E)).tocsr()
    r = linprog(c.astype(float), A_eq=A, b_eq=2 * np.ones(n), bounds=(0, 1), method="highs")
    assert r.status == 0
    return r.fun


def brute_force_opt(xy):
    """min cost over half-integral x on K_n (Section 4: the optimum is {0, 1/2, 1} valued)."""
    n = len(xy)
    row_ptr, col = complete_csr(n)
    u, v, c = edge_list(np.asarray(xy), row_ptr, col)
    E = u.size
    best = [math.inf]
    need = [4] * n  # in half units

    def rec(i, acc):
        if acc >= best[0]:
            return
        if i == E:
            if all(x == 0 for x in need):
                best[0] = acc
            return
        a, b = u[i], v[i]
        # prune: remaining edges at a node must still be able to fill it
        for val in (0, 1, 2):
            if need[a] >= val and need[b] >= val:
                need[a] -= val
                need[b] -= val
                ok = True
                if i + 1 < E:
                    # every node whose last edge is i must be full
                    for w in (a, b):
                        last = max(j for j in range(E) if u[j] == w or v[j] == w)
                        if last == i and need[w] != 0:
                            ok = False
                if ok:
                    rec(i + 1, acc + val * int(c[i]))
                need[a] += val
                need[b] += val

    rec(0, 0)
    return best[0] / 2.0


# ---- costs -----------------------------------------------------------------

def test_nint_sqrt_exhaustive_small(oracle_lib):
    d2 = np.arange(0, 1 << 22, dtype=np.int64)
    want = (_isqrt_exact(4 * d2) + 1) // 2
    assert np.array_equal(oracle_lib.nint_sqrt(d2), want)


def test_nint_sqrt_adversarial(oracle_lib):
    # d2 = r^2 + r sits just below (r + 1/2)^2, d2 = r^2 + r + 1 just above
    r = np.arange(1, 1_500_001, dtype=np.int64)
    assert np.array_equal(oracle_lib.nint_sqrt(r * r + r), r)
    assert np.array_equal(oracle_lib.nint_sqrt(r * r + r + 1), r + 1)
    # the largest distance in [0, 2^20)^2
    big = np.array([2 * (2 ** 20 - 1) ** 2], dtype=np.int64)
    assert oracle_lib.nint_sqrt(big)[0] == (_isqrt_exact(4 * big) + 1)[0] // 2


def test_nint_sqrt_random(oracle_lib):
    rng = np.random.default_rng(1)
    d2 = rng.integers(0, 2 * (2 ** 20) ** 2, size=2_000_000, dtype=np.int64)
    assert np.array_equal(oracle_lib.nint_sqrt(d2), (_isqrt_exact(4 * d2) + 1) // 2)


# ---- hand-worked sweep (Eq. 9, Eq. 10) ---------------------------------------

def test_golden_rectangle(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "rectangle_3x4.json")))
    xy = np.array(g["xy"], dtype=np.int32)
    rp, col = complete_csr(4)
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam1, b2, ch = oracle_lib.sweep(rp, col, cost, np.zeros(4, np.int32), 8, 2)
    assert st == 0 and list(lam1) == g["lambda_after_sweep1"]
    assert b2 == g["bound2_per_sweep"][0] and ch == g["changed_per_sweep"][0]
    st, lam, it, tb, tc = oracle_lib.gdp(rp, col, cost, np.zeros(4, np.int32), 8, 2, 100, trace=True)
    assert st == 0 and it == g["iterations"]
    assert list(tb) == g["bound2_per_sweep"] and list(tc) == g["changed_per_sweep"]
    bad, x2 = oracle_lib.extract(rp, col, cost, lam, 8)
    assert bad == 0
    src = np.repeat(np.arange(4), 3)
    side = np.abs(src - col) != 2  # 0-2 and 1-3 are the diagonals
    assert np.all(x2[side] == 2 * g["x_sides"]) and np.all(x2[~side] == 2 * g["x_diagonals"])
    r = oracle_lib.solve(xy, rp, col)
    assert r.certified == 2 and r.opt == g["opt"]


# ---- optimum value against independent solvers -------------------------------

@pytest.mark.parametrize("n,seed", [(4, 0), (5, 1), (5, 2), (6, 3), (6, 4)])
def test_brute_force_tiny(oracle_lib, n, seed):
    rng = np.random.default_rng(seed)
    xy = rng.integers(0, 50, size=(n, 2)).astype(np.int32)
    rp, col = complete_csr(n)
    r = oracle_lib.solve(xy, rp, col)
    assert r.status == 0 and r.certified == 2
    assert r.opt == brute_force_opt(xy)


@pytest.mark.parametrize("n,seed,side", [(12, 0, 100), (40, 1, 10 ** 6), (80, 2, 1000), (150, 3, 10 ** 6)])
def test_complete_graph_vs_highs(oracle_lib, n, seed, side):
    rng = np.random.default_rng(seed)
    xy = rng.integers(0, side + 1, size=(n, 2)).astype(np.int32)
    rp, col = complete_csr(n)
    r = oracle_lib.solve(xy, rp, col)
    assert r.status == 0 and r.certified == 2
    assert abs(r.opt - highs_opt(xy, rp, col)) < 1e-6 * max(1.0, r.opt)
    assert oracle_lib.certify(xy, r.row_ptr, r.col, r.x2, r.lam, r.frac_bits, r.bound2) == 0


@pytest.mark.parametrize("kind,n,k", [("uniform", 300, 10), ("mixture", 400, 10), ("uniform", 250, 4)])
def test_candidate_graph_with_pricing_vs_complete_highs(oracle_lib, kind, n, k):
    inst = I.make_instance(kind, n, 5, k)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    r = oracle_lib.solve(xy, rp, col)
    assert r.status == 0 and r.certified == 2
    krp, kcol = complete_csr(n)
    assert abs(r.opt - highs_opt(xy, krp, kcol)) < 1e-6 * r.opt
    assert oracle_lib.certify(xy, r.row_ptr, r.col, r.x2, r.lam, r.frac_bits, r.bound2) == 0


@pytest.mark.parametrize("kind", ["uniform", "mixture"])
def test_config_n1000_certified(oracle_lib, kind):
    inst = I.make_instance(kind, 1000, 0, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    r = oracle_lib.solve(xy, rp, col)
    assert r.status == 0 and r.certified == 2
    assert oracle_lib.certify(xy, r.row_ptr, r.col, r.x2, r.lam, r.frac_bits, r.bound2) == 0
    assert abs(r.opt - highs_opt(xy, r.row_ptr, r.col)) < 1e-6 * r.opt


# ---- closed forms --------------------------------------------------------------

@pytest.mark.parametrize("m,s,k", [(6, 7, 8), (8, 1000, 8), (10, 3, 6)])
def test_closed_form_even_grid(oracle_lib, m, s, k):
    # an even m x m grid with spacing s has a Hamiltonian cycle of unit steps and
    # every node's two shortest edges have length s, so OPT = n * s
    g = np.array([(i * s, j * s) for i in range(m) for j in range(m)], dtype=np.int32)
    rp, col = I.knn_csr(g, k)
    r = oracle_lib.solve(g, rp, col)
    assert r.status == 0 and r.certified == 2
    assert r.opt == m * m * s


def test_closed_form_two_far_triangles(oracle_lib):
    xy = np.array([[0, 0], [30, 0], [10, 40], [900000, 900000], [900050, 900000], [900020, 900070]],
                  dtype=np.int32)
    rp, col = complete_csr(6)
    r = oracle_lib.solve(xy, rp, col)
    per = lambda a, b, c: sum(round(math.dist(p, q)) for p, q in ((a, b), (b, c), (c, a)))
    assert r.certified == 2 and r.opt == per(*xy[:3]) + per(*xy[3:])


# ---- weak duality and the fixed point -----------------------------------------

def test_bound_below_opt_every_sweep(oracle_lib):
    inst = I.make_instance("uniform", 500, 3, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam, it, tb, tc = oracle_lib.gdp(rp, col, cost, np.zeros(500, np.int32), 8, 2, 20000, trace=True)
    assert st == 0
    opt = highs_opt(xy, rp, col)
    assert np.all(tb / 512.0 <= opt + 1e-9)
    # the bound climbs from 0 to within 1e-5 of the optimum
    assert tb[0] == 0 and tb[-1] / 512.0 > opt * (1 - 1e-5)
    # the last sweep changes nothing; the one before changes something
    assert tc[-1] == 0 and (it == 1 or tc[-2] > 0)


def test_fixed_point_straddles_zero(oracle_lib):
    # Section 3: at the optimum the b-th and (b+1)-th smallest adjusted values
    # straddle zero; at a GDP fixed point every node has |z(2) + z(3)| < 2^shift
    inst = I.make_instance("mixture", 600, 4, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam, it, _, _ = oracle_lib.gdp(rp, col, cost, np.zeros(600, np.int32), 8, 2, 20000)
    assert st == 0
    src = np.repeat(np.arange(600), np.diff(rp))
    z = (cost.astype(np.int64) << 8) - lam[src] - lam[col]
    for v in range(600):
        zz = np.sort(z[rp[v]:rp[v + 1]])
        assert abs(int(zz[1]) + int(zz[2])) < 4


def test_full_step_does_not_settle(oracle_lib):
    # the undamped centring step (shift 1) oscillates under Jacobi updates
    inst = I.make_instance("uniform", 300, 0, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    st, *_ = oracle_lib.gdp(rp, col, cost, np.zeros(300, np.int32), 8, 1, 3000)
    assert st == oracle_lib.OR_NOT_CONVERGED


# ---- finisher, pricing, merge ---------------------------------------------------

def test_finisher_reaches_candidate_optimum(oracle_lib):
    inst = I.make_instance("uniform", 2000, 2, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam, it, _, _ = oracle_lib.gdp(rp, col, cost, np.zeros(2000, np.int32), 8, 2, 50000)
    bad, _ = oracle_lib.extract(rp, col, cost, lam, 8)
    assert bad > 0  # the sign rule alone is not enough here
    fst, x2, lam2, aug = oracle_lib.finisher(rp, col, cost, lam, 8)
    assert fst == 0 and aug > 0
    b2 = oracle_lib.bound2(rp, col, cost, lam2, 9)
    assert oracle_lib.certify(xy, rp, col, x2, lam2, 9, b2, full_scan=False) == 0
    assert abs(b2 / 1024.0 - highs_opt(xy, rp, col)) < 1e-6 * b2 / 1024.0
    # started from lambda = 0 it reaches the same optimum
    fst0, x20, lam20, aug0 = oracle_lib.finisher(rp, col, cost, np.zeros(2000, np.int32), 8)
    assert fst0 == 0 and oracle_lib.bound2(rp, col, cost, lam20, 9) == b2 and aug0 > aug


@pytest.mark.parametrize("kind,n,seed", [("uniform", 9000, 3), ("mixture", 7000, 4)])
def test_finisher_reaches_candidate_optimum_larger(oracle_lib, kind, n, seed):
    inst = I.make_instance(kind, n, seed, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam, it, _, _ = oracle_lib.gdp(rp, col, cost, np.zeros(n, np.int32), 8, 2, 100000)
    bad, _ = oracle_lib.extract(rp, col, cost, lam, 8)
    fst, x2, lam2, aug = oracle_lib.finisher(rp, col, cost, lam, 8)
    assert fst == 0 and aug >= bad // 2 > 0
    b2 = oracle_lib.bound2(rp, col, cost, lam2, 9)
    assert oracle_lib.certify(xy, rp, col, x2, lam2, 9, b2, full_scan=False) == 0
    assert abs(b2 / 1024.0 - highs_opt(xy, rp, col)) < 1e-6 * b2 / 1024.0


def _initial_excess(rp, col, cost, lam, F, b=2):
    """Units the finisher must move: with the arcs of z < 0 saturated, node v's
    left copy holds b - #{z < 0 in row v} and its right copy the negative of
    that (z is symmetric), so the total positive excess is sum |b - that count|."""
    n = rp.size - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    z = (cost.astype(np.int64) << F) - lam[src].astype(np.int64) - lam[col]
    neg = np.bincount(src[z < 0], minlength=n)
    return int(np.abs(b - neg).sum())


def test_finisher_certified_from_a_short_gdp(oracle_lib):
    # 40,000 nodes, lambda after 64 sweeps leaves many rows off.  The
    # certificate (x feasible, complementary slackness, equal cost and bound)
    # proves the result optimal on the graph; every augmentation moves one unit
    # of the initial excess; the finisher from lambda = 0 reaches the same optimum.
    inst = I.make_instance("uniform", 40000, 6, 6)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam, it, _, _ = oracle_lib.gdp(rp, col, cost, np.zeros(40000, np.int32), 8, 2, 64)
    bad, _ = oracle_lib.extract(rp, col, cost, lam, 8)
    fst, x2, lam2, aug = oracle_lib.finisher(rp, col, cost, lam, 8)
    assert fst == 0 and aug >= bad // 2 > 1000
    assert aug == _initial_excess(rp, col, cost, lam, 8)
    b2 = oracle_lib.bound2(rp, col, cost, lam2, 9)
    assert oracle_lib.certify(xy, rp, col, x2, lam2, 9, b2, full_scan=False) == 0
    fst0, x20, lam20, aug0 = oracle_lib.finisher(rp, col, cost, np.zeros(40000, np.int32), 8)
    assert fst0 == 0 and oracle_lib.bound2(rp, col, cost, lam20, 9) == b2
    assert aug0 == _initial_excess(rp, col, cost, np.zeros(40000, np.int32), 8)


def test_finisher_infeasible_graph(oracle_lib):
    # K_{3,5}: the five right nodes need 10 units of x, the three left nodes supply 6
    xy = np.array([[0, 0], [0, 10], [0, 20]] + [[100, 7 * i] for i in range(5)], dtype=np.int32)
    rows = [[3, 4, 5, 6, 7]] * 3 + [[0, 1, 2]] * 5
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    cost = oracle_lib.cost_table(xy, rp, col)
    st, *_ = oracle_lib.finisher(rp, col, cost, np.zeros(8, np.int32), 8)
    assert st == oracle_lib.OR_INFEASIBLE


def test_pricing_matches_all_pairs(oracle_lib):
    inst = I.make_instance("mixture", 700, 1, 6)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    rng = np.random.default_rng(0)
    lam = rng.integers(0, 40000 * 256, size=700).astype(np.int32)
    for fb in (8, 9):
        cnt, pairs = oracle_lib.pricing(xy, rp, col, lam, fb)
        # independent: every pair, exact integer cost, minus the CSR edges
        iu, iv = np.triu_indices(700, 1)
        d = xy[iu].astype(np.int64) - xy[iv]
        c = (_isqrt_exact(4 * (d[:, 0] ** 2 + d[:, 1] ** 2)) + 1) // 2
        neg = (c << fb) - lam[iu].astype(np.int64) - lam[iv] < 0
        src = np.repeat(np.arange(700), np.diff(rp))
        incsr = set(zip(src.tolist(), col.tolist()))
        want = [(a, b) for a, b in zip(iu[neg].tolist(), iv[neg].tolist()) if (a, b) not in incsr]
        assert cnt == len(want) > 0
        assert [tuple(p) for p in pairs.tolist()] == want


def test_merge_is_sorted_union(oracle_lib):
    inst = I.make_instance("uniform", 200, 1, 4)
    rp, col = inst["row_ptr"], inst["col"]
    pairs = np.array([[0, 150], [3, 7], [3, 199], [10, 11]], dtype=np.int32)
    nrp, ncl = oracle_lib.merge(rp, col, pairs)
    src = np.repeat(np.arange(200), np.diff(rp))
    want = set(zip(src.tolist(), col.tolist()))
    for a, b in pairs.tolist():
        want.add((a, b)); want.add((b, a))
    want = sorted(want)
    nsrc = np.repeat(np.arange(200), np.diff(nrp))
    assert list(zip(nsrc.tolist(), ncl.tolist())) == want


# ---- certificate: planted mistakes are caught -----------------------------------

def test_certificate_catches_planted_mistakes(oracle_lib):
    inst = I.make_instance("uniform", 400, 7, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    r = oracle_lib.solve(xy, rp, col)
    ok = lambda x2, lam, b2, fb=r.frac_bits: oracle_lib.certify(xy, r.row_ptr, r.col, x2, lam, fb, b2)
    assert ok(r.x2, r.lam, r.bound2) == 0
    x2 = r.x2.copy(); x2[np.argmax(x2 == 2)] = 0
    assert ok(x2, r.lam, r.bound2) != 0           # one x dropped
    lam = r.lam.copy(); lam[5] += 10 ** 7
    assert ok(r.x2, lam, r.bound2) != 0           # one dual moved far: slackness breaks
    assert ok(r.x2, r.lam, r.bound2 + 1) != 0     # bound off by one unit
    assert ok(r.x2, r.lam * 2, r.bound2 * 2, r.frac_bits + 1) == 0  # same point, finer grid
    # lambda raised everywhere: some outside pair turns negative -> check 7
    big = r.lam + (2000 << r.frac_bits)
    assert oracle_lib.certify(xy, r.row_ptr, r.col, r.x2, big, r.frac_bits, 0, True) != 0


# ---- metamorphic ------------------------------------------------------------------

def test_node_permutation_and_translation(oracle_lib):
    inst = I.make_instance("uniform", 500, 9, 10)
    xy, rp, col = inst["xy"], inst["row_ptr"], inst["col"]
    cost = oracle_lib.cost_table(xy, rp, col)
    st, lam, it, tb, _ = oracle_lib.gdp(rp, col, cost, np.zeros(500, np.int32), 8, 2, 20000, trace=True)
    perm = np.random.default_rng(3).permutation(500)
    inv = np.argsort(perm)
    pxy = xy[perm]  # new node i is old node perm[i]
    prp, pcol = I.knn_csr(pxy, 10)
    pcost = oracle_lib.cost_table(pxy, prp, pcol)
    # same graph relabelled (the kNN lists can differ only through index tie-breaks)
    src = np.repeat(np.arange(500), np.diff(rp))
    psrc = np.repeat(np.arange(500), np.diff(prp))
    if set(zip(inv[src].tolist(), inv[col].tolist())) == set(zip(psrc.tolist(), pcol.tolist())):
        st2, lam2, it2, tb2, _ = oracle_lib.gdp(prp, pcol, pcost, np.zeros(500, np.int32), 8, 2, 20000, trace=True)
        assert it2 == it and np.array_equal(lam2, lam[perm]) and np.array_equal(tb2, tb)
    # integer translation and swapping x with y change no cost
    for t in (xy + 1234, xy[:, ::-1].copy()):
        c2 = oracle_lib.cost_table(t.astype(np.int32), rp, col)
        assert np.array_equal(c2, cost)
