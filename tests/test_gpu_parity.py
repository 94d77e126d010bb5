"""CUDA path vs the CPU oracle, through the C ABI.

Steps covered bit for bit: cost table (a1), GDP sweeps with their per-sweep
bound and changed count (a2-a5), sign extraction (a6), pricing scan (a7), CSR
merge (a8), and the whole solve up to the finisher (lambda, x, bound,
iteration and round counts).  From the finisher on, the optimum, the
certification and the certificate (see parity_helpers.py: optimal lambda and x
are not unique).  Sizes span several tiles of every kernel with ragged tails;
the full-size workloads are checked on sampled outputs and, solved whole,
against stored records of the oracle's solves of the same instances.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from paper_2011_08170_gb300 import build as B
from parity_helpers import compare_solves, same_optimum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def inst(kind, n, seed, k):
    return I.make_instance(kind, n, seed, k)


def complete_csr(n):
    rp = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int32)
    col = np.array([j for i in range(n) for j in range(n) if j != i], dtype=np.int32)
    return rp, col


CASES = [("uniform", 1000, 0, 10), ("mixture", 2500, 3, 10), ("uniform", 777, 5, 6),
         ("mixture", 5000, 1, 12)]


# ---- a1: cost table ---------------------------------------------------------------

@pytest.mark.parametrize("kind,n,seed,k", CASES)
def test_cost_table(lib, O, kind, n, seed, k):
    d = inst(kind, n, seed, k)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    rp, col, x2, cost = f2m.f2m_get_x(ctx)
    assert np.array_equal(rp, d["row_ptr"]) and np.array_equal(col, d["col"])
    assert np.array_equal(cost, O.cost_table(d["xy"], d["row_ptr"], d["col"]))


def test_cost_extremes(lib, O):
    # corners of [0, 2^20)^2, duplicate points, and distances near half-integers
    M = (1 << 20) - 1
    xy = np.array([[0, 0], [M, M], [0, M], [M, 0], [0, 0], [3, 4], [1000, 1001], [M, M - 1]],
                  dtype=np.int32)
    rp, col = complete_csr(8)
    ctx = f2m.f2m_create(xy, rp, col)
    _, _, _, cost = f2m.f2m_get_x(ctx)
    assert np.array_equal(cost, O.cost_table(xy, rp, col))


# ---- a2-a5: GDP sweeps ------------------------------------------------------------------

# flags 0: shared-memory tiled kernel, two sweeps per barrier; 2: the same, one
# sweep per barrier; 1: streaming kernel
@pytest.mark.parametrize("flags", [0, 1, 2])
@pytest.mark.parametrize("kind,n,seed,k", CASES)
def test_gdp_phase_trace(lib, O, kind, n, seed, k, flags):
    d = inst(kind, n, seed, k)
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    st_o, lam_o, it_o, tb_o, tc_o = O.gdp(d["row_ptr"], d["col"], cost, np.zeros(n, np.int32),
                                          8, 2, 100000, trace=True)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(flags=flags))
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 100000, trace_cap=it_o)
    lam, fb = f2m.f2m_get_lambda(ctx)
    assert (st == f2m.F2M_OK) == (st_o == O.OR_OK)
    assert sweeps == it_o and fb == 8
    assert np.array_equal(lam, lam_o)
    assert np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)


@pytest.mark.parametrize("flags", [0, 1, 2])
@pytest.mark.parametrize("shift", [1, 2, 3])
def test_single_sweeps_from_random_lambda(lib, O, shift, flags):
    d = inst("mixture", 3000, 7, 10)
    n = 3000
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    rng = np.random.default_rng(shift)
    params = f2m.f2m_default_params(damping_shift=shift, flags=flags)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], params)
    for trial in range(3):
        lam = rng.integers(-(1 << 24), 1 << 24, size=n).astype(np.int32)
        f2m.f2m_set_lambda(ctx, lam, 8)
        st_o, lam_o, b2_o, ch_o = O.sweep(d["row_ptr"], d["col"], cost, lam, 8, shift)
        st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 1, trace_cap=1)
        out, _ = f2m.f2m_get_lambda(ctx)
        assert sweeps == 1 and np.array_equal(out, lam_o)
        assert tb[0] == b2_o and tc[0] == ch_o


def test_golden_rectangle_on_gpu(lib, O):
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rectangle_3x4.json")))
    xy = np.array(g["xy"], dtype=np.int32)
    rp, col = complete_csr(4)
    ctx = f2m.f2m_create(xy, rp, col)
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 100, trace_cap=10)
    assert st == f2m.F2M_OK and sweeps == g["iterations"]
    assert list(tb) == g["bound2_per_sweep"] and list(tc) == g["changed_per_sweep"]
    info = f2m.f2m_solve(ctx)
    assert info.certified == 2 and info.bound2 / (2 * (1 << info.frac_bits)) == g["opt"]


# ---- a6: extraction ----------------------------------------------------------------------

@pytest.mark.parametrize("fb", [8, 9])
def test_extraction(lib, O, fb):
    d = inst("uniform", 2000, 4, 10)
    n = 2000
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    _, lam, *_ = O.gdp(d["row_ptr"], d["col"], cost, np.zeros(n, np.int32), 8, 2, 100000)
    if fb == 9:
        lam = lam * 2 + np.random.default_rng(0).integers(-1, 2, size=n).astype(np.int32)
    bad_o, x2_o = O.extract(d["row_ptr"], d["col"], cost, lam, fb)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_set_lambda(ctx, lam, fb)
    bad, x2 = f2m.f2m_extract(ctx)
    assert bad == bad_o and np.array_equal(x2, x2_o)


# ---- a7: pricing --------------------------------------------------------------------------

def _sorted_pairs(p):
    p = np.asarray(p).reshape(-1, 2)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


# pricing 1: full scan; 2: the scan with far tile pairs skipped (same pairs)
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("kind,n,seed,k,fb", [("mixture", 2500, 1, 6, 8), ("uniform", 3333, 2, 4, 9),
                                              ("uniform", 1024, 3, 5, 8), ("mixture", 1025, 4, 5, 8),
                                              ("mixture", 20000, 5, 6, 8)])
def test_pricing_random_lambda(lib, O, kind, n, seed, k, fb, mode):
    d = inst(kind, n, seed, k)
    rng = np.random.default_rng(seed)
    scale = 30000 if kind == "uniform" else 8000
    lam = rng.integers(-scale, scale * 3, size=n).astype(np.int32) << fb
    lam = (lam + rng.integers(0, 1 << fb, size=n)).astype(np.int32)
    cnt_o, pairs_o = O.pricing(d["xy"], d["row_ptr"], d["col"], lam, fb)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(pricing=mode))
    f2m.f2m_set_lambda(ctx, lam, fb)
    cnt, pairs = f2m.f2m_price(ctx)
    assert cnt == cnt_o > 0
    assert np.array_equal(_sorted_pairs(pairs), pairs_o)


@pytest.mark.parametrize("mode", [1, 2])
def test_pricing_boundary_z_minus_one_and_zero(lib, O, mode):
    # lambdas set so that many outside pairs have z exactly 0 or -1: the fp32
    # filter must keep every z = -1 pair and the exact test must drop z = 0
    n = 2048
    d = inst("uniform", n, 11, 4)
    xy = d["xy"]
    rng = np.random.default_rng(5)
    fb = 8
    lam = np.zeros(n, np.int64)
    # pair node 2i with node 2i+1: lam split so that lam_u + lam_v = c*2^fb + {0, 1}
    for i in range(0, n - 1, 2):
        c = int(O.nint_sqrt(np.array([int(((xy[i] - xy[i + 1]).astype(np.int64) ** 2).sum())]))[0])
        tot = (c << fb) + (i // 2) % 2
        a = int(rng.integers(0, tot + 1))
        lam[i], lam[i + 1] = a, tot - a
    lam = lam.astype(np.int32)
    cnt_o, pairs_o = O.pricing(xy, d["row_ptr"], d["col"], lam, fb)
    ctx = f2m.f2m_create(xy, d["row_ptr"], d["col"], f2m.f2m_default_params(pricing=mode))
    f2m.f2m_set_lambda(ctx, lam, fb)
    cnt, pairs = f2m.f2m_price(ctx)
    assert cnt == cnt_o and cnt > 0
    assert np.array_equal(_sorted_pairs(pairs), pairs_o)


@pytest.mark.parametrize("mode", [1, 2])
def test_pricing_nothing_to_find(lib, O, mode):
    d = inst("uniform", 1500, 2, 10)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(pricing=mode))
    cnt, _ = f2m.f2m_price(ctx)  # lambda = 0: every z >= 0
    assert cnt == 0


@pytest.mark.parametrize("mode", [1, 2])
def test_pricing_buffer_grows(lib, O, mode):
    d = inst("uniform", 1200, 3, 4)
    n = 1200
    lam = np.full(n, 200000 << 8, dtype=np.int32)  # every pair negative
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(pricing_cap=16, pricing=mode))
    f2m.f2m_set_lambda(ctx, lam, 8)
    cnt, pairs = f2m.f2m_price(ctx)
    cnt_o, pairs_o = O.pricing(d["xy"], d["row_ptr"], d["col"], lam, 8)
    assert cnt == cnt_o and np.array_equal(_sorted_pairs(pairs), pairs_o)


# ---- a8: merge -----------------------------------------------------------------------------

def test_merge(lib, O):
    d = inst("mixture", 3000, 9, 6)
    rng = np.random.default_rng(1)
    u = rng.integers(0, 3000, size=5000)
    v = rng.integers(0, 3000, size=5000)
    keep = u != v
    pairs = np.stack([np.minimum(u, v), np.maximum(u, v)], 1)[keep].astype(np.int32)
    pairs = np.unique(pairs, axis=0)
    rp_o, col_o = O.merge(d["row_ptr"], d["col"], pairs)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_add_edges(ctx, pairs[rng.permutation(len(pairs))])
    rp, col, _, cost = f2m.f2m_get_x(ctx)
    assert np.array_equal(rp, rp_o) and np.array_equal(col, col_o)
    assert np.array_equal(cost, O.cost_table(d["xy"], rp_o, col_o))
    # adding pairs already present (either direction) changes nothing
    f2m.f2m_add_edges(ctx, pairs[:100, ::-1].copy())
    rp2, col2, _, _ = f2m.f2m_get_x(ctx)
    assert np.array_equal(rp2, rp_o) and np.array_equal(col2, col_o)


def test_read_back_into_caller_buffers(lib):
    # the out= forms write the same values into the caller's arrays (pinned
    # host tensors, numpy arrays with spare room) and return their leading parts
    import torch
    d = inst("uniform", 5000, 4, 10)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_solve(ctx)
    rp, col, x2, cost = f2m.f2m_get_x(ctx)
    lam, fb = f2m.f2m_get_lambda(ctx)
    m = len(col)
    pinned = (torch.empty(5001, dtype=torch.int32).pin_memory(), torch.empty(m + 7, dtype=torch.int32).pin_memory(),
              torch.empty(m + 7, dtype=torch.uint8).pin_memory(), torch.empty(m + 7, dtype=torch.int32).pin_memory())
    plain = (np.full(5003, -1, np.int32), np.full(m, -1, np.int32), np.full(m + 1, 9, np.uint8),
             np.full(m + 2, -1, np.int32))
    for out in (pinned, plain):
        got = f2m.f2m_get_x(ctx, out=out)
        for a, b in zip(got, (rp, col, x2, cost)):
            assert np.array_equal(np.asarray(a), b)
    lam_out = torch.empty(5000, dtype=torch.int32).pin_memory()
    got, fb2 = f2m.f2m_get_lambda(ctx, out=lam_out)
    assert fb2 == fb and np.array_equal(got.numpy(), lam)
    with pytest.raises(f2m.F2MError):  # room for fewer entries than the graph has: INVALID_ARG
        f2m.f2m_get_x(ctx, out=(plain[0], plain[1][:m - 1], plain[2], plain[3]))
    with pytest.raises(ValueError):  # a row_ptr array too short is caught before the call
        f2m.f2m_get_x(ctx, out=(plain[0][:5000], plain[1], plain[2], plain[3]))


def test_merge_sequence_touching_few_rows(lib, O):
    # rows no pair touches are carried over as they are: merges of a few
    # pairs, one of pairs already present, then one that outgrows the edge
    # arrays, each equal to the oracle's union of everything added so far
    n = 20000
    d = inst("uniform", n, 3, 10)
    rng = np.random.default_rng(7)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    rp_o, col_o = d["row_ptr"], d["col"]
    present = np.stack([np.repeat(np.arange(n), np.diff(rp_o))[:5], col_o[:5]], 1).astype(np.int32)
    for size in (3, 40, 0, 2 * len(col_o)):
        if size == 0:
            pairs = present
        else:
            u = rng.integers(0, n, size=size)
            v = rng.integers(0, n, size=size)
            keep = u != v
            pairs = np.stack([u, v], 1)[keep].astype(np.int32)
        rp_o, col_o = O.merge(rp_o, col_o, np.unique(np.sort(pairs, 1), axis=0))
        f2m.f2m_add_edges(ctx, pairs)
        rp, col, _, cost = f2m.f2m_get_x(ctx)
        assert np.array_equal(rp, rp_o) and np.array_equal(col, col_o)
        assert np.array_equal(cost, O.cost_table(d["xy"], rp_o, col_o))


# ---- the whole solve ------------------------------------------------------------------------

def _compare_solve(O, d, **kw):
    mi = kw.get("max_iters", 1000000)
    return compare_solves(O, f2m, d,
                          params=dict(max_iters=mi, flags=kw.get("flags", 0), pricing=kw.get("pricing", 1)),
                          oracle_kw=dict(max_iters=mi))


@pytest.mark.parametrize("flags", [0, 1, 2])
@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 1000, 0, 10), ("mixture", 1000, 0, 10),
                                           ("mixture", 3000, 2, 10), ("uniform", 2000, 1, 6)])
def test_solve_bit_exact(lib, O, kind, n, seed, k, flags):
    s, r = _compare_solve(O, inst(kind, n, seed, k), flags=flags)
    assert s.info["certified"] == 2


@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 2000, 1, 6), ("mixture", 5000, 3, 4)])
def test_solve_bit_exact_with_culled_pricing(lib, O, kind, n, seed, k):
    s, r = _compare_solve(O, inst(kind, n, seed, k), pricing=2)
    assert s.info["certified"] == 2


# GDP phases cut at max_iters sweeps (tiny, odd, the default 128 and 256): the solve
# goes on from the lambda reached, bit-exact with the oracle all the way
@pytest.mark.parametrize("flags", [0, 1, 2])
@pytest.mark.parametrize("cap", [1, 7, 64, 128, 256])
@pytest.mark.parametrize("kind,n,seed,k", [("mixture", 3000, 2, 10), ("uniform", 2000, 1, 6)])
def test_solve_bit_exact_with_capped_phases(lib, O, kind, n, seed, k, cap, flags):
    s, r = _compare_solve(O, inst(kind, n, seed, k), max_iters=cap, flags=flags)
    assert s.info["certified"] == 2 and s.info["iterations"] <= cap * s.info["phases"]


def test_default_solve_equals_oracle_default(lib, O):
    # both sides at their defaults (128 sweeps per phase); a sparse graph that
    # takes several phases and pricing rounds
    d = inst("mixture", 5000, 3, 4)
    assert f2m.f2m_default_params().max_iters == 128
    s, r = compare_solves(O, f2m, d)
    assert r.phases > 1 and s.info["certified"] == 2


@pytest.mark.parametrize("kind,n,seed,k,rows", [("uniform", 20000, 0, 10, True), ("mixture", 20000, 1, 12, True),
                                                ("mixture", 9000, 3, 4, False)])
def test_certifying_scan_of_the_finisher_lambda(lib, O, kind, n, seed, k, rows):
    # after a finisher call the scan of its lambda covers only the rows whose
    # lambda rose (a pair elsewhere stays z >= 0): fewer pairs than a full
    # scan; the solve matches the oracle's (which scans in full) up to the
    # finisher bit for bit and after it by its optimum, and the oracle's
    # certificate -- its own scan of all n(n-1)/2 pairs -- accepts the result
    # (rows False: a sparse graph whose last GDP phase follows the last
    # complete scan, so the finisher's lambda is scanned in full)
    d = inst(kind, n, seed, k)
    s, r = compare_solves(O, f2m, d)
    assert s.info["certified"] == 2 and s.info["finisher_calls"] >= 1
    full = n * (n - 1) // 2
    if rows:
        assert s.info["certifying_scans"] >= 1
        assert s.info["pricing_pairs"] < s.info["pricing_rounds"] * full
    else:
        assert s.info["certifying_scans"] == 0
        assert s.info["pricing_pairs"] == s.info["pricing_rounds"] * full
    # a context whose lambda is then set by hand scans in full again
    ctx = f2m.f2m_create(d["xy"], s.row_ptr, s.col)
    f2m.f2m_set_lambda(ctx, s.lam, s.frac_bits)
    cnt, _ = f2m.f2m_price(ctx)
    assert cnt == 0


@pytest.mark.parametrize("flags", [0, 2])
def test_gdp_after_a_solve_that_merged(lib, O, flags):
    # a solve whose scans added edges ends with the finisher's lambda (F + 1
    # bits) on the merged graph; a GDP phase called afterwards starts from the
    # floor to F bits on that graph, like the oracle's
    d = inst("mixture", 5000, 3, 4)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(flags=flags))
    info = f2m.f2m_solve(ctx)
    assert info.edges_added > 0 and info.frac_bits == 9
    lam9, _ = f2m.f2m_get_lambda(ctx)
    rp, col, _, cost = f2m.f2m_get_x(ctx)
    st_o, lam_o, it_o, tb_o, tc_o = O.gdp(rp, col, cost, lam9 >> 1, 8, 2, 50, trace=True)
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 50, trace_cap=50)
    assert sweeps == it_o and np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)
    assert np.array_equal(f2m.f2m_get_lambda(ctx)[0], lam_o)


def _full_size_records():
    path = os.path.join(os.path.dirname(__file__), "golden", "full_size_solves.json")
    return json.load(open(path)) if os.path.exists(path) else {}


FULL = _full_size_records()


def _digest(a, dt):
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dt).tobytes()).hexdigest()


@pytest.mark.parametrize("name", sorted(FULL))
def test_full_size_solve_equals_oracle_record(lib, O, name):
    # the 100,000- and 200,000-point workloads solved whole, against the
    # oracle's records of the same solves (written by
    # golden/make_full_size_solves.py): bit for bit up to the finisher, then
    # the same optimum, certified
    g = FULL[name]
    d = inst(g["kind"], g["n"], g["seed"], g["k"])
    bf = g["before_finisher"]
    s0 = f2m.solve(d["xy"], d["row_ptr"], d["col"], raise_on_error=False,
                   params=f2m.f2m_default_params(max_iters=g["max_iters"], finisher=0))
    for k in ("status", "iterations", "phases", "pricing_rounds", "edges_added", "bound2", "frac_bits", "nnz"):
        assert s0.info[k] == bf[k], ("before the finisher", k, s0.info[k], bf[k])
    got = {"row_ptr": _digest(s0.row_ptr, "<i4"), "col": _digest(s0.col, "<i4"), "x2": _digest(s0.x2, "u1"),
           "lam": _digest(s0.lam, "<i4")}
    assert got == bf["sha256"]

    sv = g["solve"]
    s = f2m.solve(d["xy"], d["row_ptr"], d["col"], params=f2m.f2m_default_params(max_iters=g["max_iters"]))
    i = s.info
    assert i["status"] == sv["status"] == 0 and i["certified"] == sv["certified"] == 2
    assert same_optimum(i["bound2"], i["frac_bits"], sv["bound2"], sv["frac_bits"])
    if i["finisher_calls"] == sv["finisher_calls"] == 1:
        assert i["augmentations"] == sv["augmentations"]
    # the certificate on the candidate graph (x feasible, slackness, cost =
    # bound), and no negative pair in a sample of rows of the complete graph
    assert O.certify(d["xy"], s.row_ptr, s.col, s.x2, s.lam, s.frac_bits, i["bound2"], full_scan=False) == 0
    n = g["n"]
    for u0 in np.random.default_rng(1).choice(n - 256, 4, replace=False):
        cnt, _ = O.pricing(d["xy"], s.row_ptr, s.col, s.lam, s.frac_bits, rows=(int(u0), int(u0) + 256))
        assert cnt == 0


def test_solve_complete_graph_small(lib, O):
    rng = np.random.default_rng(3)
    xy = rng.integers(0, 1000, size=(40, 2)).astype(np.int32)
    rp, col = complete_csr(40)
    _compare_solve(O, {"xy": xy, "row_ptr": rp, "col": col})


def test_solve_warm_start_and_resume(lib, O):
    d = inst("uniform", 1500, 8, 10)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    st, sweeps, *_ = f2m.f2m_gdp(ctx, 200)
    lam_mid, fb = f2m.f2m_get_lambda(ctx)
    # resume in a new context from the checkpoint: same as running straight on
    a = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_gdp(a, 200)
    f2m.f2m_gdp(a, 100000)
    b = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_set_lambda(b, lam_mid, fb)
    f2m.f2m_gdp(b, 100000)
    assert np.array_equal(f2m.f2m_get_lambda(a)[0], f2m.f2m_get_lambda(b)[0])
    info = f2m.f2m_solve(b)
    r = O.solve(d["xy"], d["row_ptr"], d["col"], lam0=lam_mid)
    assert same_optimum(info.bound2, info.frac_bits, r.bound2, r.frac_bits) and info.certified == 2
    compare_solves(O, f2m, d, lam0=lam_mid)


# ---- error paths (no fault: statuses only) --------------------------------------------------

def test_invalid_csr_rejected(lib):
    d = inst("uniform", 300, 0, 6)
    rp, col, xy = d["row_ptr"].copy(), d["col"].copy(), d["xy"].copy()
    bad = []
    c1 = col.copy(); c1[rp[5]] = 5; bad.append((xy, rp, c1, "self-loop"))
    c2 = col.copy(); c2[rp[7]], c2[rp[7] + 1] = c2[rp[7] + 1], c2[rp[7]]; bad.append((xy, rp, c2, "sorted"))
    x3 = xy.copy(); x3[3, 0] = 1 << 20; bad.append((x3, rp, col, "coordinate"))
    c4 = col.copy(); c4[rp[9]] = 299 if c4[rp[9]] != 299 else 298; bad.append((xy, rp, c4, ""))
    for x, r, c, word in bad:
        with pytest.raises(f2m.F2MError) as e:
            f2m.f2m_create(x, r, c)
        assert e.value.status == f2m.F2M_ERR_INVALID_ARG and word in str(e.value)


def test_iteration_cap_gives_not_converged(lib):
    d = inst("uniform", 1000, 0, 10)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    st, sweeps, *_ = f2m.f2m_gdp(ctx, 3)
    assert st == f2m.F2M_ERR_NOT_CONVERGED and sweeps == 3


def test_overflow_status(lib, O):
    d = inst("uniform", 1000, 0, 10)
    n = 1000
    # node 0 high, its neighbours low: its adjusted lengths stay at c * 2^F and
    # the update pushes lambda_0 past 2^29 on the first sweep
    lam = np.zeros(n, dtype=np.int32)
    lam[0] = (1 << 29) - 5
    lam[d["col"][d["row_ptr"][0]:d["row_ptr"][1]]] = -(1 << 29) + 5
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    f2m.f2m_set_lambda(ctx, lam, 8)
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 10, trace_cap=10)
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    st_o, lam_o, it_o, tb_o, tc_o = O.gdp(d["row_ptr"], d["col"], cost, lam, 8, 2, 10, trace=True)
    assert st == f2m.F2M_ERR_OVERFLOW and st_o == O.OR_OVERFLOW and sweeps == it_o
    assert np.array_equal(f2m.f2m_get_lambda(ctx)[0], lam_o)
    with pytest.raises(f2m.F2MError):
        f2m.f2m_set_lambda(ctx, np.full(n, 1 << 29, np.int32), 8)


def test_overflow_in_either_sweep_of_a_round(lib, O):
    # K_{3,7} has no fractional 2-matching: GDP raises lambda without bound and
    # overflows after 6,607,469 sweeps (oracle).  Starting 10 or 11 sweeps
    # before that (the oracle's state there) puts the overflow in the second or
    # the first sweep of a two-sweep round; both kernels must stop exactly where
    # the oracle does, with the oracle's lambda and traces.
    m = 7
    xy = np.array([[0, 0], [0, 10], [0, 20]] + [[100, 7 * i] for i in range(m)], dtype=np.int32)
    rows = [list(range(3, 3 + m))] * 3 + [[0, 1, 2]] * m
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    cost = O.cost_table(xy, rp, col)
    st_full, _, it_full, _, _ = O.gdp(rp, col, cost, np.zeros(len(xy), np.int32), 8, 2, 10 ** 7, trace=False)
    assert st_full == O.OR_OVERFLOW and it_full == 6607470
    for back in (10, 11):
        st0, lam0, it0, _, _ = O.gdp(rp, col, cost, np.zeros(len(xy), np.int32), 8, 2, it_full - back, trace=False)
        assert st0 == O.OR_NOT_CONVERGED
        st_o, lam_o, it_o, tb_o, tc_o = O.gdp(rp, col, cost, lam0, 8, 2, 50, trace=True)
        assert st_o == O.OR_OVERFLOW and it_o == back
        for flags in (0, 2):
            ctx = f2m.f2m_create(xy, rp, col, f2m.f2m_default_params(flags=flags, pricing=0))
            f2m.f2m_set_lambda(ctx, lam0, 8)
            st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 50, trace_cap=50)
            assert st == f2m.F2M_ERR_OVERFLOW and sweeps == it_o, (back, flags, st, sweeps)
            assert np.array_equal(f2m.f2m_get_lambda(ctx)[0], lam_o), (back, flags)
            assert np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)


def test_barrier_wait_budget_runs_out_and_context_recovers(lib):
    # a zero spin budget makes every non-last block give up at its first
    # barrier: the kernel returns a TIMEOUT status instead of waiting
    d = inst("uniform", 20000, 0, 10)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"], f2m.f2m_default_params(barrier_budget_cycles=0))
    st, sweeps, *_ = f2m.f2m_gdp(ctx, 50)
    assert st == f2m.F2M_ERR_TIMEOUT
    ok = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    st, sweeps, *_ = f2m.f2m_gdp(ok, 5)
    assert st == f2m.F2M_ERR_NOT_CONVERGED and sweeps == 5


def test_infeasible_candidate_graph(lib):
    # K_{3,5}: right side needs 10 units, left side offers 6.  GDP pushes lambda
    # of the right nodes up without bound; either the overflow guard or the
    # finisher reports it.
    xy = np.array([[0, 0], [0, 10], [0, 20]] + [[100, 7 * i] for i in range(5)], dtype=np.int32)
    rows = [[3, 4, 5, 6, 7]] * 3 + [[0, 1, 2]] * 5
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    ctx = f2m.f2m_create(xy, rp, col, f2m.f2m_default_params(pricing=0, max_iters=2000))
    info = f2m.f2m_solve(ctx, raise_on_error=False)
    assert info.status in (f2m.F2M_ERR_INFEASIBLE, f2m.F2M_ERR_OVERFLOW)


def test_tiled_path_on_tiny_and_clustered_graphs(lib, O):
    # few nodes per CTA, duplicate points, dense clusters: renumbering ties and
    # halos that cover most of the graph
    rng = np.random.default_rng(9)
    xy = np.concatenate([rng.integers(0, 50, size=(300, 2)), rng.integers(0, 10 ** 6, size=(200, 2)),
                         np.repeat([[777, 777]], 12, axis=0)]).astype(np.int32)
    rp, col = I.knn_csr(xy, 8)
    cost = O.cost_table(xy, rp, col)
    st_o, lam_o, it_o, tb_o, tc_o = O.gdp(rp, col, cost, np.zeros(len(xy), np.int32), 8, 2, 100000, trace=True)
    ctx = f2m.f2m_create(xy, rp, col)
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 100000, trace_cap=it_o)
    assert sweeps == it_o and np.array_equal(f2m.f2m_get_lambda(ctx)[0], lam_o)
    assert np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)
    _compare_solve(O, {"xy": xy, "row_ptr": rp, "col": col})


def test_gdp_full_size_sampled(lib, O):
    # the 100,000-node workload: the first 40 sweeps bit-exact against the
    # oracle, then the fixed point checked node by node on a sample
    d = inst("uniform", 100000, 0, 10)
    n = 100000
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    st_o, lam_o, it_o, tb_o, tc_o = O.gdp(d["row_ptr"], d["col"], cost, np.zeros(n, np.int32),
                                          8, 2, 40, trace=True)
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    st, sweeps, tb, tc = f2m.f2m_gdp(ctx, 40, trace_cap=40)
    assert sweeps == 40 and np.array_equal(f2m.f2m_get_lambda(ctx)[0], lam_o)
    assert np.array_equal(tb, tb_o) and np.array_equal(tc, tc_o)
    st, sweeps, *_ = f2m.f2m_gdp(ctx, 10 ** 6)
    assert st == f2m.F2M_OK
    lam, _ = f2m.f2m_get_lambda(ctx)
    rp, col = d["row_ptr"], d["col"]
    for v in np.random.default_rng(0).choice(n, 300, replace=False):
        row = slice(rp[v], rp[v + 1])
        z = np.sort((cost[row].astype(np.int64) << 8) - lam[v] - lam[col[row]])
        assert abs(int(z[1]) + int(z[2])) < 4  # a fixed point of the update
    # one more oracle sweep from the GPU fixed point changes nothing
    st1, lam1, b2, ch = O.sweep(rp, col, cost, lam, 8, 2)
    assert ch == 0 and np.array_equal(lam1, lam)


def test_two_sweep_packed_entries_at_full_size(lib, O):
    # the 200,000-point clustered workload (k = 12): the 8-byte two-sweep tiles
    # do not fit shared memory, the packed (4-byte) ones do.  The packed
    # kernel's sweeps equal the one-sweep kernel's, and its last sweep equals
    # the oracle's sweep from the GPU's previous lambda.
    d = inst("mixture", 200000, 0, 12)
    rp, col = d["row_ptr"], d["col"]
    p0 = f2m.f2m_default_params(pricing=0, finisher=0, max_iters=60)
    info = f2m.f2m_solve(f2m.f2m_create(d["xy"], rp, col, p0), raise_on_error=False)
    assert info.gdp_kernel == f2m.F2M_GDP_KERNEL_TWO_SWEEP_PACKED and info.iterations == 60
    runs = {}
    for flags in (0, f2m.F2M_FLAG_ONE_SWEEP_GDP):
        ctx = f2m.f2m_create(d["xy"], rp, col, f2m.f2m_default_params(flags=flags))
        _, sw1, tb, tc = f2m.f2m_gdp(ctx, 59, trace_cap=59)
        lam59, _ = f2m.f2m_get_lambda(ctx)
        f2m.f2m_gdp(ctx, 1)
        lam60, _ = f2m.f2m_get_lambda(ctx)
        runs[flags] = (sw1, tb, tc, lam59, lam60)
    a, b = runs[0], runs[f2m.F2M_FLAG_ONE_SWEEP_GDP]
    assert a[0] == b[0] == 59
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    cost = O.cost_table(d["xy"], rp, col)
    st, lam_o, _, _ = O.sweep(rp, col, cost, a[3], 8, 2)
    assert st == O.OR_OK and np.array_equal(lam_o, a[4])
