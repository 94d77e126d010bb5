"""Degree requirements b_v (fractional b-matching, Section 3 with Eq. 8) on the
CUDA path vs the CPU oracle, through the C ABI.  Every comparison is bit-exact,
except that whole solves are compared bit for bit up to the finisher and by
their optimum after it (parity_helpers.py).

Covers both selection methods of the streaming GDP kernel (registers when every
b_v < 8, counting otherwise), the bound and rule (7) extraction with b, the
finisher's b_v supplies, the whole solve with pricing, and the argument checks
of f2m_set_degrees.
"""
import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from parity_helpers import compare_solves
from paper_2011_08170_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def complete_csr(n):
    rp = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int32)
    col = np.array([j for i in range(n) for j in range(n) if j != i], dtype=np.int32)
    return rp, col


def random_b(rp, lo, hi, seed):
    """b_v uniform in [lo, hi], capped at deg(v) - 1."""
    deg = np.diff(rp)
    b = np.random.default_rng(seed).integers(lo, hi + 1, size=deg.size)
    return np.minimum(b, deg - 1).astype(np.int32)


# (kind, n, seed, k, b range): b < 8 runs on registers, larger b by counting
CASES = [("uniform", 1000, 0, 10, (1, 4)), ("mixture", 2500, 3, 10, (1, 3)),
         ("uniform", 777, 5, 6, (1, 5)), ("mixture", 3000, 1, 12, (1, 11)),
         ("uniform", 1500, 2, 16, (6, 14))]


# flags 0: the two-sweep shared-memory kernel; 1: the streaming kernel
@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("kind,n,seed,k,br", CASES)
def test_gdp_phase_trace_with_b(lib, O, kind, n, seed, k, br, flags):
    d = I.make_instance(kind, n, seed, k)
    b = random_b(d["row_ptr"], *br, seed)
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    st_o, lam_o, it_o, tb_o, tc_o = O.gdp(d["row_ptr"], d["col"], cost, np.zeros(n, np.int32),
                                          8, 2, 100000, trace=True, b=b)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(flags=flags))
    f2m.f2m_set_degrees(ctx, b)
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 100000, trace_cap=it_o)
    lam, fb = f2m.f2m_get_lambda(ctx)
    assert (st == f2m.F2M_OK) == (st_o == O.OR_OK)
    assert sweeps == it_o
    assert np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)
    assert np.array_equal(lam, lam_o)


@pytest.mark.parametrize("kind,n,seed,k,br", CASES[:3])
def test_bound_and_extract_with_b(lib, O, kind, n, seed, k, br):
    d = I.make_instance(kind, n, seed, k)
    b = random_b(d["row_ptr"], *br, seed + 7)
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    lam = np.random.default_rng(seed).integers(0, 5000 * 256, size=n).astype(np.int32)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_set_degrees(ctx, b)
    f2m.f2m_set_lambda(ctx, lam, 8)
    b2, fb = f2m.f2m_get_bound(ctx)
    assert fb == 8 and b2 == O.bound2(d["row_ptr"], d["col"], cost, lam, 8, b=b)
    bad, x2 = f2m.f2m_extract(ctx)
    bad_o, x2_o = O.extract(d["row_ptr"], d["col"], cost, lam, 8, b=b)
    assert bad == bad_o and np.array_equal(x2, x2_o)


def _compare_solve_b(O, d, b, **kw):
    pricing = kw.get("pricing", 1)
    return compare_solves(O, f2m, d, b=b, params=dict(max_iters=1000000, pricing=pricing),
                          oracle_kw=dict(max_iters=1000000, pricing=pricing != 0))


# b vectors for which the b-matching LP is feasible on the candidate graph
SOLVE_CASES = [("uniform", 1000, 0, 10, (1, 4)), ("mixture", 2500, 3, 10, (1, 3)),
               ("uniform", 777, 5, 6, (2, 4)), ("mixture", 3000, 1, 12, (8, 10)),
               ("uniform", 1500, 2, 16, (6, 14))]


@pytest.mark.parametrize("kind,n,seed,k,br", SOLVE_CASES)
def test_solve_with_b_bit_exact(lib, O, kind, n, seed, k, br):
    d = I.make_instance(kind, n, seed, k)
    b = random_b(d["row_ptr"], *br, seed + 1)
    s, r = _compare_solve_b(O, d, b)
    assert s.info["certified"] == 2
    assert O.certify(d["xy"], s.row_ptr, s.col, s.x2, s.lam, s.frac_bits, s.info["bound2"], b=b) == 0


@pytest.mark.parametrize("kind,n,seed,k,br", [("uniform", 777, 5, 6, (1, 5)),
                                              ("mixture", 3000, 1, 12, (1, 11))])
@pytest.mark.parametrize("flags", [0, 1])
def test_infeasible_candidate_graph_overflows_alike(lib, O, kind, n, seed, k, br, flags):
    # these b have no fractional b-matching on the k-NN graph: the dual is
    # unbounded and both sides stop at |lambda| = 2^29 after the same sweeps
    d = I.make_instance(kind, n, seed, k)
    b = random_b(d["row_ptr"], *br, seed + 1)
    r = O.solve(d["xy"], d["row_ptr"], d["col"], max_iters=1000000, b=b)
    assert r.status == O.OR_OVERFLOW
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(max_iters=1000000, flags=flags))
    f2m.f2m_set_degrees(ctx, b)
    info = f2m.f2m_solve(ctx, raise_on_error=False)
    assert info.status == f2m.F2M_ERR_OVERFLOW and info.iterations == r.iterations


@pytest.mark.parametrize("pricing", [1, 2])
def test_solve_with_b_and_pricing_modes(lib, O, pricing):
    d = I.make_instance("mixture", 4000, 9, 5)
    b = random_b(d["row_ptr"], 1, 3, 4)
    s, r = _compare_solve_b(O, d, b, pricing=pricing)
    assert s.info["edges_added"] > 0


def test_complete_graph_b_near_degree(lib, O):
    # K_40 with b = 38 = deg - 1 (counting path) and b = 1
    rng = np.random.default_rng(5)
    xy = rng.integers(0, 3000, size=(40, 2)).astype(np.int32)
    rp, col = complete_csr(40)
    d = {"xy": xy, "row_ptr": rp, "col": col}
    for bval in (38, 1, 20):
        _compare_solve_b(O, d, np.full(40, bval, np.int32))


def test_b2_through_set_degrees_equals_default(lib, O):
    # b = 2 everywhere runs on the streaming degree kernel, not the tiled one;
    # the result must not change
    d = I.make_instance("uniform", 3000, 4, 10)
    a = f2m.solve(d["xy"], d["row_ptr"], d["col"])
    c = f2m.solve(d["xy"], d["row_ptr"], d["col"], b=2)
    for k in ("iterations", "bound2", "frac_bits", "certified", "finisher_calls"):
        assert a.info[k] == c.info[k], k
    assert np.array_equal(a.lam, c.lam) and np.array_equal(a.x2, c.x2)


def test_set_degrees_checks_and_reset(lib, O):
    d = I.make_instance("uniform", 500, 6, 6)
    rp = d["row_ptr"]
    ctx = f2m.f2m_create(d["xy"], rp, d["col"])
    b = random_b(rp, 1, 3, 0)
    f2m.f2m_set_degrees(ctx, b)
    bad = b.copy()
    bad[123] = int(rp[124] - rp[123])  # needs degree b + 1
    with pytest.raises(f2m.F2MError) as ei:
        f2m.f2m_set_degrees(ctx, bad)
    assert ei.value.status == f2m.F2M_ERR_INVALID_ARG and "123" in str(ei.value)
    bad[123] = 0
    with pytest.raises(f2m.F2MError):
        f2m.f2m_set_degrees(ctx, bad)
    # the previous b stays
    cost = O.cost_table(d["xy"], rp, d["col"])
    st, sweeps, *_ = f2m.f2m_gdp(ctx, 100000)
    st_o, lam_o, it_o, _, _ = O.gdp(rp, d["col"], cost, np.zeros(500, np.int32), 8, 2, 100000, b=b)
    lam, _ = f2m.f2m_get_lambda(ctx)
    assert sweeps == it_o and np.array_equal(lam, lam_o)
    # None restores b = 2
    f2m.f2m_set_degrees(ctx, None)
    f2m.f2m_set_lambda(ctx, np.zeros(500, np.int32), 8)
    f2m.f2m_gdp(ctx, 100000)
    lam2, _ = f2m.f2m_get_lambda(ctx)
    _, lam2_o, _, _, _ = O.gdp(rp, d["col"], cost, np.zeros(500, np.int32), 8, 2, 100000)
    assert np.array_equal(lam2, lam2_o)


def test_infeasible_b(lib, O):
    # K_{3,5} plus nothing else: with b = 1 on the left and b = 1 on the right the
    # five right nodes need 5 units, the three left nodes supply 3 -> infeasible
    xy = np.array([[0, 0], [0, 10], [0, 20]] + [[100, 7 * i] for i in range(5)], dtype=np.int32)
    rows = [[3, 4, 5, 6, 7]] * 3 + [[0, 1, 2]] * 5
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    b = np.ones(8, np.int32)
    r = O.solve(xy, rp, col, b=b, pricing=False, max_iters=2000)
    assert r.status == O.OR_INFEASIBLE
    ctx = f2m.f2m_create(xy, rp, col, f2m.f2m_default_params(pricing=0, max_iters=2000))
    f2m.f2m_set_degrees(ctx, b)
    info = f2m.f2m_solve(ctx, raise_on_error=False)
    assert info.status == f2m.F2M_ERR_INFEASIBLE
