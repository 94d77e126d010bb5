"""Subtour-elimination cuts on the CUDA path vs the CPU oracle (oracle/subtour.c),
through the C ABI.  Every comparison is bit-exact.

Covers the separation (components of the support of x as one cut layer),
GDP sweeps over node and cut duals with their per-sweep bound and changed
count (one and several layers), the bound and rule (7) with the cut terms,
pricing with the cut terms, the whole driver f2m_solve_subtour (stages of GDP
and pricing with layers added between them), the overflow status, and the
argument checks of f2m_add_cut_layer.
"""
import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from paper_2011_08170_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def _layers_from_oracle(O, d, rounds):
    """The oracle's cut family after `rounds` rounds of its driver, and the
    lambda its stage 0 reached (the start of the cut phases below)."""
    r0 = O.solve_subtour(d["xy"], d["row_ptr"], d["col"], rounds=0, pricing=False)
    r = O.solve_subtour(d["xy"], d["row_ptr"], d["col"], rounds=rounds, pricing=False)
    return r0, r


@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 1000, 0, 10), ("mixture", 2500, 3, 10),
                                           ("uniform", 777, 5, 6)])
def test_separation_equals_oracle(lib, O, kind, n, seed, k):
    d = I.make_instance(kind, n, seed, k)
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    st, lam, *_ = O.gdp(d["row_ptr"], d["col"], cost, np.zeros(n, np.int32), 8, 2, 300)
    _, x2 = O.extract(d["row_ptr"], d["col"], cost, lam, 8)
    comp_o, m_o = O.separate(d["row_ptr"], d["col"], x2)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_set_lambda(ctx, lam, 8)
    f2m.f2m_extract(ctx)
    comp, m = f2m.f2m_separate(ctx)
    assert m == m_o > 3 and np.array_equal(comp, comp_o)


@pytest.mark.parametrize("layers", [1, 3])
@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 1200, 1, 10), ("mixture", 2000, 2, 8)])
def test_cut_gdp_trace_equals_oracle(lib, O, kind, n, seed, k, layers):
    d = I.make_instance(kind, n, seed, k)
    rp, col = d["row_ptr"], d["col"]
    cost = O.cost_table(d["xy"], rp, col)
    r0, r = _layers_from_oracle(O, d, layers)
    cuts = r.cuts
    assert cuts.L == layers
    st_o, lam_o, mu_o, it_o, tb_o, tc_o = O.cut_gdp(rp, col, cost, cuts, r0.lam, None, 8, 2, 700, trace=True)
    ctx = f2m.f2m_create(d["xy"], rp, col)
    f2m.f2m_set_lambda(ctx, r0.lam, 8)
    for l in range(cuts.L):
        f2m.f2m_add_cut_layer(ctx, cuts.comp[l], int(cuts.ncuts[l]))
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 700, trace_cap=it_o)
    lam, fb = f2m.f2m_get_lambda(ctx)
    mu, nl = f2m.f2m_get_cut_duals(ctx)
    assert (st == f2m.F2M_OK) == (st_o == O.OR_OK) and sweeps == it_o and fb == 8 and nl == layers
    assert np.array_equal(lam, lam_o) and np.array_equal(mu, mu_o)
    assert np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)
    # bound and rule (7) with the cut terms at the duals reached
    b2, _ = f2m.f2m_get_bound(ctx)
    assert b2 == O.cut_bound2(rp, col, cost, cuts, lam_o, mu_o, 8)
    bad, x2 = f2m.f2m_extract(ctx)
    bad_o, x2_o = O.cut_extract(rp, col, cost, cuts, lam_o, mu_o, 8)
    assert bad == bad_o and np.array_equal(x2, x2_o)
    # a phase cut short and resumed equals one phase
    a = f2m.f2m_create(d["xy"], rp, col)
    f2m.f2m_set_lambda(a, r0.lam, 8)
    for l in range(cuts.L):
        f2m.f2m_add_cut_layer(a, cuts.comp[l], int(cuts.ncuts[l]))
    f2m.f2m_gdp(a, 37)
    f2m.f2m_gdp(a, 700 - 37)
    if sweeps == 700:
        assert np.array_equal(f2m.f2m_get_lambda(a)[0], lam_o)
        assert np.array_equal(f2m.f2m_get_cut_duals(a)[0], mu_o)


def test_cut_pricing_equals_oracle(lib, O):
    d = I.make_instance("uniform", 3000, 4, 5)
    rp, col = d["row_ptr"], d["col"]
    cost = O.cost_table(d["xy"], rp, col)
    r0, r = _layers_from_oracle(O, d, 2)
    st_o, lam_o, mu_o, it_o, _, _ = O.cut_gdp(rp, col, cost, r.cuts, r0.lam, None, 8, 2, 400)
    ctx = f2m.f2m_create(d["xy"], rp, col)
    f2m.f2m_set_lambda(ctx, r0.lam, 8)
    for l in range(r.cuts.L):
        f2m.f2m_add_cut_layer(ctx, r.cuts.comp[l], int(r.cuts.ncuts[l]))
    f2m.f2m_gdp(ctx, 400)
    # raise lambda so that many outside pairs turn negative
    rng = np.random.default_rng(3)
    lam = lam_o + rng.integers(0, 3000 * 256, size=3000).astype(np.int32)
    f2m.f2m_set_lambda(ctx, lam, 8)
    cnt_o, pairs_o = O.cut_pricing(d["xy"], rp, col, r.cuts, lam, mu_o, 8)
    cnt, pairs = f2m.f2m_price(ctx)
    assert cnt == cnt_o > 100
    got = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    assert np.array_equal(got, pairs_o)


@pytest.mark.parametrize("kind,n,seed,k,rounds", [("uniform", 1500, 0, 10, 3), ("mixture", 2500, 1, 10, 4),
                                                  ("uniform", 800, 7, 5, 2)])
def test_solve_subtour_equals_oracle(lib, O, kind, n, seed, k, rounds):
    d = I.make_instance(kind, n, seed, k)
    r = O.solve_subtour(d["xy"], d["row_ptr"], d["col"], rounds=rounds)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    info = f2m.f2m_solve_subtour(ctx, rounds)
    for key in ("iterations", "phases", "pricing_rounds", "edges_added", "cuts", "bound2_f2m", "bound2",
                "rounds", "layers", "frac_bits", "certified", "status"):
        assert info[key] == r.info[key], (key, info[key], r.info[key])
    assert info["status"] == 0 and info["rounds"] >= 1 and info["bound2"] > info["bound2_f2m"]
    lam, _ = f2m.f2m_get_lambda(ctx)
    mu, layers = f2m.f2m_get_cut_duals(ctx)
    rp, col, x2, _ = f2m.f2m_get_x(ctx)
    assert np.array_equal(lam, r.lam) and np.array_equal(mu, r.mu) and layers == r.cuts.L
    assert np.array_equal(rp, r.row_ptr) and np.array_equal(col, r.col) and np.array_equal(x2, r.x2)


def test_cut_overflow_status(lib, O):
    # node 0 high and its neighbours low: its update passes 2^29 in the first
    # sweep of the phase with cuts; both sides stop there with the input state
    d = I.make_instance("uniform", 1000, 0, 10)
    rp, col = d["row_ptr"], d["col"]
    cost = O.cost_table(d["xy"], rp, col)
    r0, r = _layers_from_oracle(O, d, 1)
    lam0 = r0.lam.copy()
    lam0[0] = (1 << 29) - 5
    lam0[col[rp[0]:rp[1]]] = -(1 << 29) + 5
    st_o, lam_o, mu_o, it_o, tb_o, tc_o = O.cut_gdp(rp, col, cost, r.cuts, lam0, None, 8, 2, 50, trace=True)
    ctx = f2m.f2m_create(d["xy"], rp, col, f2m.f2m_default_params(pricing=0))
    f2m.f2m_set_lambda(ctx, lam0, 8)
    f2m.f2m_add_cut_layer(ctx, r.cuts.comp[0], int(r.cuts.ncuts[0]))
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 50, trace_cap=50)
    assert st_o == O.OR_OVERFLOW and st == f2m.F2M_ERR_OVERFLOW and sweeps == it_o
    assert np.array_equal(f2m.f2m_get_lambda(ctx)[0], lam_o)
    assert np.array_equal(f2m.f2m_get_cut_duals(ctx)[0], mu_o)
    assert np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)


def test_add_cut_layer_checks(lib, O):
    d = I.make_instance("uniform", 600, 2, 8)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    comp = np.full(600, -1, np.int32)
    comp[:10] = 0
    comp[20] = 3  # outside [-1, ncuts)
    with pytest.raises(f2m.F2MError) as e:
        f2m.f2m_add_cut_layer(ctx, comp, 2)
    assert e.value.status == f2m.F2M_ERR_INVALID_ARG and "node 20" in str(e.value)
    assert f2m.f2m_get_cut_duals(ctx)[1] == 0
    # a single node's cut is its own star: fine; a cut that only 2 candidate
    # edges leave is refused and the context keeps no layer
    comp = np.full(600, -1, np.int32)
    comp[5] = 0
    f2m.f2m_add_cut_layer(ctx, comp, 1)
    assert f2m.f2m_get_cut_duals(ctx)[1] == 1
    with pytest.raises(f2m.F2MError):
        f2m.f2m_solve(ctx)  # the F2M solve loop refuses a context with cuts
    xy = np.array([[0, 0], [0, 9], [9, 0], [9, 9], [50, 0], [50, 9], [59, 0], [59, 9]], np.int32)
    nb = [[1, 2, 3, 4], [0, 2, 3, 5], [0, 1, 3], [0, 1, 2], [0, 5, 6, 7], [1, 4, 6, 7], [4, 5, 7], [4, 5, 6]]
    rp2 = np.concatenate([[0], np.cumsum([len(x) for x in nb])]).astype(np.int32)
    col2 = np.array([c for x in nb for c in sorted(x)], np.int32)
    c2 = f2m.f2m_create(xy, rp2, col2)
    with pytest.raises(f2m.F2MError) as e:
        f2m.f2m_add_cut_layer(c2, np.array([0, 0, 0, 0, -1, -1, -1, -1], np.int32), 1)
    assert "fewer than 3" in str(e.value)
    assert f2m.f2m_get_cut_duals(c2)[1] == 0
