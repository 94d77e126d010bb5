"""Whole-solve comparison of the CUDA library with the CPU oracle.

A solve has two kinds of steps.

(i) Steps with one exact result: every GDP phase (Eq. 9, Eq. 10), every pricing
scan, every merge and the sign rule (7).  Both sides run the same integer
algorithm, so with the finisher switched off -- the solve then stops at the
first extraction that leaves a row off, or ends certified without one -- the
counters, the candidate graph, lambda, x and the bound agree bit for bit.

(ii) The exact finisher (Section 3, last paragraph: the repair of a degenerate
stop is left to the problem).  The oracle runs one plain sequential
successive-shortest-path search; the library runs blocks of it on host
threads.  Both end at an optimal flow with optimal potentials, but optimal
lambda and x are not unique, so from the finisher on only what is unique is
compared: the optimum (bound2 at frac_bits, as a rational), the certification
level, and -- where each side called the finisher once, from the same state --
the number of unit augmentations (the initial excess, which each augmentation
lowers by one).  The library's result must also pass the oracle's independent
certificate (feasible x, complementary slackness, cost = bound, and with
pricing no negative pair anywhere in the complete graph).
"""
import numpy as np

BEFORE_FINISHER_KEYS = ("status", "iterations", "phases", "pricing_rounds", "edges_added", "bound2",
                        "frac_bits", "certified")


def same_optimum(b2a, fba, b2b, fbb):
    """bound2 / 2^fb equal as rationals."""
    return int(b2a) << int(fbb) == int(b2b) << int(fba)


def compare_solves(O, f2m, d, b=None, lam0=None, params=None, oracle_kw=None):
    """(i) bit-exact with the finisher off, then (ii) result parity with it on.

    params: keyword overrides of f2m_default_params; oracle_kw: keyword
    arguments of oracle.solve describing the same solve.  Returns the library's
    and the oracle's complete solves."""
    params = dict(params or {})
    oracle_kw = dict(oracle_kw or {})
    xy, rp, col = d["xy"], d["row_ptr"], d["col"]

    r0 = O.solve(xy, rp, col, b=b, lam0=lam0, finisher=False, **oracle_kw)
    s0 = f2m.solve(xy, rp, col, lam0=lam0, b=b, raise_on_error=False,
                   params=f2m.f2m_default_params(**dict(params, finisher=0)))
    for k in BEFORE_FINISHER_KEYS:
        assert s0.info[k] == getattr(r0, k), ("before the finisher", k, s0.info[k], getattr(r0, k))
    assert np.array_equal(s0.row_ptr, r0.row_ptr) and np.array_equal(s0.col, r0.col)
    assert np.array_equal(s0.lam, r0.lam) and np.array_equal(s0.x2, r0.x2)

    r = O.solve(xy, rp, col, b=b, lam0=lam0, **oracle_kw)
    s = f2m.solve(xy, rp, col, lam0=lam0, b=b, params=f2m.f2m_default_params(**params))
    i = s.info
    assert i["status"] == r.status == 0
    assert i["certified"] == r.certified
    assert same_optimum(i["bound2"], i["frac_bits"], r.bound2, r.frac_bits), (i["bound2"], r.bound2)
    if r0.status == O.OR_OK:
        # no row was off: no finisher ran and the whole solve is case (i)
        assert i["finisher_calls"] == r.finisher_calls == 0
        for k in ("iterations", "phases", "pricing_rounds", "edges_added", "bound2", "frac_bits"):
            assert i[k] == getattr(r, k), k
        assert np.array_equal(s.lam, r.lam) and np.array_equal(s.x2, r.x2)
    else:
        assert i["finisher_calls"] >= 1 and r.finisher_calls >= 1
        if i["finisher_calls"] == r.finisher_calls == 1:
            assert i["augmentations"] == r.augmentations
    full = oracle_kw.get("pricing", True) and params.get("pricing", 1) != 0
    assert O.certify(xy, s.row_ptr, s.col, s.x2, s.lam, s.frac_bits, i["bound2"], full_scan=full,
                     b=b) == 0
    return s, r
