"""Class-by-class (Gauss-Seidel) GDP on the CUDA path vs the CPU oracle,
through the C ABI.  Every comparison is bit-exact, except that whole solves
are compared bit for bit up to the finisher and by their optimum after it
(parity_helpers.py).

Covers the Jones-Plassmann colouring against the oracle's sequential greedy
colouring (including more than 64 colours), per-sweep traces and lambda for
both step sizes and all three row-selection forms, the overflow rule, and whole
solves with pricing (the colouring is redone after each merge).
"""
import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from parity_helpers import compare_solves
from paper_2011_08170_gb300 import build as B

pytestmark = pytest.mark.gpu

GS = f2m.F2M_FLAG_CLASS_SWEEPS


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


@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 1000, 0, 10), ("mixture", 5000, 3, 10),
                                           ("uniform", 777, 5, 6), ("mixture", 20000, 1, 16)])
def test_colouring_matches_sequential_greedy(lib, O, kind, n, seed, k):
    d = I.make_instance(kind, n, seed, k)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    nc, color = f2m.f2m_get_colors(ctx)
    nc_o, color_o = O.color_greedy(d["row_ptr"], d["col"])
    assert nc == nc_o and np.array_equal(color, color_o)


def test_colouring_complete_graph_past_64_colours(lib, O):
    rng = np.random.default_rng(2)
    xy = rng.integers(0, 10000, size=(100, 2)).astype(np.int32)
    rp, col = complete_csr(100)
    ctx = f2m.f2m_create(xy, rp, col)
    nc, color = f2m.f2m_get_colors(ctx)
    nc_o, color_o = O.color_greedy(rp, col)
    assert nc == nc_o == 100 and np.array_equal(color, color_o)


def _b(rp, lo, hi, seed):
    deg = np.diff(rp)
    return np.minimum(np.random.default_rng(seed).integers(lo, hi + 1, size=deg.size), deg - 1).astype(np.int32)


@pytest.mark.parametrize("shift", [1, 2])
@pytest.mark.parametrize("kind,n,seed,k,br", [("uniform", 1000, 0, 10, None), ("mixture", 2500, 3, 10, None),
                                              ("uniform", 777, 5, 6, None), ("mixture", 3000, 1, 12, (1, 4)),
                                              ("uniform", 1500, 2, 16, (6, 12))])
def test_class_phase_trace(lib, O, kind, n, seed, k, br, shift):
    d = I.make_instance(kind, n, seed, k)
    rp, col = d["row_ptr"], d["col"]
    b = None if br is None else _b(rp, *br, seed)
    cost = O.cost_table(d["xy"], rp, col)
    nc, color = O.color_greedy(rp, col)
    st_o, lam_o, it_o, tb_o, tc_o = O.gdp_gs(rp, col, cost, np.zeros(n, np.int32), color, nc,
                                             8, shift, 100000, trace=True, b=b)
    ctx = f2m.f2m_create(d["xy"], rp, col, f2m.f2m_default_params(flags=GS, damping_shift=shift))
    if b is not None:
        f2m.f2m_set_degrees(ctx, b)
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 100000, trace_cap=it_o)
    lam, _ = f2m.f2m_get_lambda(ctx)
    assert (st == f2m.F2M_OK) == (st_o == O.OR_OK)
    assert sweeps == it_o and np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)
    assert np.array_equal(lam, lam_o)
    if shift == 1:
        assert np.all(np.diff(tb) >= 0)  # block coordinate ascent


def test_class_phase_untraced_and_partial(lib, O):
    # without a trace the bound pass is skipped; a phase cut short by max_sweeps
    # and resumed gives the same lambda as one long phase
    d = I.make_instance("uniform", 4000, 7, 10)
    rp, col = d["row_ptr"], d["col"]
    cost = O.cost_table(d["xy"], rp, col)
    nc, color = O.color_greedy(rp, col)
    st_o, lam_o, it_o, _, _ = O.gdp_gs(rp, col, cost, np.zeros(4000, np.int32), color, nc, 8, 2, 100000)
    ctx = f2m.f2m_create(d["xy"], rp, col, f2m.f2m_default_params(flags=GS))
    st, s1, *_ = f2m.f2m_gdp(ctx, 37)
    assert st == f2m.F2M_ERR_NOT_CONVERGED and s1 == 37
    st, s2, *_ = f2m.f2m_gdp(ctx, 100000)
    lam, _ = f2m.f2m_get_lambda(ctx)
    assert st == f2m.F2M_OK and s1 + s2 == it_o and np.array_equal(lam, lam_o)


def test_class_overflow_rule(lib, O):
    d = I.make_instance("uniform", 2000, 1, 6)
    rp, col = d["row_ptr"], d["col"]
    cost = O.cost_table(d["xy"], rp, col)
    nc, color = O.color_greedy(rp, col)
    lam0 = np.zeros(2000, np.int32)
    for v in np.nonzero(color == 0)[0][:5]:
        lam0[col[rp[v]:rp[v + 1]]] = -(1 << 29) + 64
    st_o, lam_o, it_o, _, _ = O.gdp_gs(rp, col, cost, lam0, color, nc, 8, 1, 1000)
    assert st_o == O.OR_OVERFLOW
    ctx = f2m.f2m_create(d["xy"], rp, col, f2m.f2m_default_params(flags=GS, damping_shift=1))
    f2m.f2m_set_lambda(ctx, lam0, 8)
    st, sweeps, *_ = f2m.f2m_gdp(ctx, 1000)
    lam, _ = f2m.f2m_get_lambda(ctx)
    assert st == f2m.F2M_ERR_OVERFLOW and sweeps == it_o and np.array_equal(lam, lam_o)


@pytest.mark.parametrize("kind,n,seed,k,shift,b", [("uniform", 2000, 1, 6, 2, None),
                                                   ("mixture", 3000, 2, 10, 1, None),
                                                   ("uniform", 1500, 4, 8, 2, 3)])
def test_class_solve_bit_exact(lib, O, kind, n, seed, k, shift, b):
    d = I.make_instance(kind, n, seed, k)
    s, r = compare_solves(O, f2m, d, b=b, params=dict(max_iters=1000000, flags=GS, damping_shift=shift),
                          oracle_kw=dict(max_iters=1000000, classes=True, shift=shift))
    assert s.info["certified"] == 2