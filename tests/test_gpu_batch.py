"""Batched solves: each instance of a batch equals its own single solve and is certified.

The batch runs every instance through one persistent GDP launch per phase (with
converged instances frozen), shared pricing scans, merges, extraction and
finisher calls.  Per instance, the sweep count, phases, pricing rounds, edges
added, finisher calls, optimum, lambda (scaled to a common number of
fractional bits), x and final candidate graph must equal those of f2m_solve on
that instance alone, and the oracle's certificate must accept the result.
"""
import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from parity_helpers import compare_solves, same_optimum
from paper_2011_08170_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


def make_batch(specs):
    out = []
    for kind, n, seed, k in specs:
        d = I.make_instance(kind, n, seed, k)
        out.append(d)
    return out


def compare(O, ds, params=None):
    b = f2m.f2m_create_batch([(d["xy"], d["row_ptr"], d["col"]) for d in ds], params)
    infos, tot = f2m.f2m_solve_batch(b)
    assert tot.status == 0 and tot.certified == 2
    for i, d in enumerate(ds):
        s = f2m.solve(d["xy"], d["row_ptr"], d["col"], params=params)
        bi = infos[i]
        for k in ("iterations", "phases", "pricing_rounds", "edges_added", "finisher_calls", "certified"):
            assert getattr(bi, k) == s.info[k], (i, k, getattr(bi, k), s.info[k])
        lam, fb = f2m.f2m_batch_get_lambda(b, i)
        rp, col, x2 = f2m.f2m_batch_get_x(b, i)
        fbm = max(fb, s.frac_bits)
        assert np.array_equal(lam.astype(np.int64) << (fbm - fb), s.lam.astype(np.int64) << (fbm - s.frac_bits))
        assert bi.bound2 << (fbm - fb) == s.info["bound2"] << (fbm - s.frac_bits)
        assert np.array_equal(rp, s.row_ptr) and np.array_equal(col, s.col) and np.array_equal(x2, s.x2)
        assert O.certify(d["xy"], rp, col, x2, lam, fb, bi.bound2) == 0
    return b, infos, tot


def test_batch_equals_single_solves(lib, oracle_lib):
    ds = make_batch([("uniform", 1000, 0, 10), ("mixture", 1500, 1, 10), ("uniform", 300, 2, 10),
                     ("mixture", 2200, 3, 10), ("uniform", 777, 4, 6), ("uniform", 2048, 5, 10)])
    compare(oracle_lib, ds)


def test_batch_with_pricing_rounds_and_waiting_instances(lib, oracle_lib):
    # small k forces pricing pairs (extra GDP phases) in some instances while
    # others wait; some need the finisher, some not
    ds = make_batch([("uniform", 600, 11, 4), ("mixture", 900, 12, 10), ("uniform", 1200, 13, 5),
                     ("mixture", 400, 14, 4), ("uniform", 1000, 0, 10)])
    b, infos, tot = compare(oracle_lib, ds)
    assert max(i.phases for i in infos) > 1 and min(i.phases for i in infos) == 1


def test_batch_with_culled_pricing(lib, oracle_lib):
    ds = make_batch([("uniform", 600, 11, 4), ("mixture", 900, 12, 10), ("uniform", 1200, 13, 5),
                     ("mixture", 400, 14, 4)])
    compare(oracle_lib, ds, f2m.f2m_default_params(pricing=2))


def test_batch_matches_oracle_optimum(lib, oracle_lib):
    # each instance of the batch: the optimum of the oracle's solve, exactly; an
    # instance that needed no finisher has the oracle's lambda and x bit for
    # bit; and the single solve that the batch equals (compare above) is the
    # oracle's, bit for bit up to the finisher and by its optimum after it
    ds = make_batch([("uniform", 800, 21, 8), ("mixture", 1100, 22, 10), ("uniform", 500, 23, 6)])
    b = f2m.f2m_create_batch([(d["xy"], d["row_ptr"], d["col"]) for d in ds])
    infos, tot = f2m.f2m_solve_batch(b)
    for i, d in enumerate(ds):
        r = oracle_lib.solve(d["xy"], d["row_ptr"], d["col"])  # both at 128 sweeps per phase
        fb = infos[i].frac_bits
        assert same_optimum(infos[i].bound2, fb, r.bound2, r.frac_bits)
        assert infos[i].certified == r.certified == 2
        lam, _ = f2m.f2m_batch_get_lambda(b, i)
        rp, col, x2 = f2m.f2m_batch_get_x(b, i)
        if r.finisher_calls == 0:
            assert infos[i].finisher_calls == 0 and fb == r.frac_bits
            assert np.array_equal(lam, r.lam) and np.array_equal(x2, r.x2)
        compare_solves(oracle_lib, f2m, d)
        # the same read into the caller's buffers (with spare room)
        n, m = len(d["xy"]), len(col)
        out = (np.zeros(n + 3, np.int32), np.zeros(m + 5, np.int32), np.zeros(m + 5, np.uint8))
        got = f2m.f2m_batch_get_x(b, i, out=out)
        assert all(np.array_equal(a, c) for a, c in zip(got, (rp, col, x2)))
        got_lam, _ = f2m.f2m_batch_get_lambda(b, i, out=np.zeros(n + 1, np.int32))
        assert np.array_equal(got_lam, lam)


def test_batch_log_uniform_sizes(lib, oracle_lib):
    # a scaled-down version of the 256-instance workload: sizes log-uniform,
    # uniform and clustered instances alternating
    rng = np.random.default_rng(7)
    specs = [("uniform" if i % 2 == 0 else "mixture", int(round(np.exp(rng.uniform(np.log(300), np.log(3000))))), i, 10)
             for i in range(24)]
    ds = make_batch(specs)
    b = f2m.f2m_create_batch([(d["xy"], d["row_ptr"], d["col"]) for d in ds])
    infos, tot = f2m.f2m_solve_batch(b)
    assert tot.status == 0 and tot.certified == 2
    for i, d in enumerate(ds):
        lam, fb = f2m.f2m_batch_get_lambda(b, i)
        rp, col, x2 = f2m.f2m_batch_get_x(b, i)
        assert oracle_lib.certify(d["xy"], rp, col, x2, lam, fb, infos[i].bound2) == 0


def test_batch_rejects_cross_instance_column(lib):
    ds = make_batch([("uniform", 300, 1, 6), ("uniform", 300, 2, 6)])
    bad = ds[1]["col"].copy()
    bad[0] = 300  # outside its instance
    with pytest.raises(f2m.F2MError) as e:
        f2m.f2m_create_batch([(ds[0]["xy"], ds[0]["row_ptr"], ds[0]["col"]),
                              (ds[1]["xy"], ds[1]["row_ptr"], bad)])
    assert e.value.status == f2m.F2M_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", list(range(12)))
def test_every_kernel_shape_gives_the_same_result(lib, oracle_lib, shape):
    # each shape of the batched GDP kernel (the autotuner's candidates): same
    # sweeps, lambda and x as the single solves
    ds = make_batch([("uniform", 700, 31, 10), ("mixture", 1300, 32, 10), ("uniform", 2100, 33, 6),
                     ("mixture", 450, 34, 10)])
    compare(oracle_lib, ds, f2m.f2m_default_params(batch_shape=shape))


def _clusters():
    return f2m.f2m_default_params(flags=f2m.F2M_FLAG_BATCH_CLUSTERS)


def test_cluster_sizes_match_single_solves(lib, oracle_lib):
    # instance sizes that take clusters of 1, 2, 4, 8 and 16 CTAs (at most 2048
    # nodes and 24,000 entries per CTA)
    ds = make_batch([("uniform", 1500, 31, 10), ("mixture", 3000, 32, 10), ("uniform", 6000, 33, 10),
                     ("mixture", 12000, 34, 10), ("uniform", 20000, 35, 10), ("uniform", 37, 36, 6)])
    compare(oracle_lib, ds, _clusters())


def test_cluster_batch_with_pricing_rounds(lib, oracle_lib):
    ds = make_batch([("uniform", 600, 11, 4), ("mixture", 900, 12, 10), ("uniform", 1200, 13, 5),
                     ("mixture", 400, 14, 4), ("uniform", 1000, 0, 10)])
    compare(oracle_lib, ds, _clusters())


def test_cluster_and_streaming_batch_paths_agree(lib):
    ds = make_batch([("uniform", 4000, 41, 10), ("mixture", 9000, 42, 8), ("uniform", 700, 43, 5)])
    res = []
    for flags in (0, f2m.F2M_FLAG_BATCH_CLUSTERS):
        b = f2m.f2m_create_batch([(d["xy"], d["row_ptr"], d["col"]) for d in ds],
                                 f2m.f2m_default_params(flags=flags))
        infos, tot = f2m.f2m_solve_batch(b)
        assert tot.status == 0
        res.append([(i.iterations, i.phases, i.bound2, f2m.f2m_batch_get_lambda(b, k)[0].tobytes(),
                     f2m.f2m_batch_get_x(b, k)[2].tobytes()) for k, i in enumerate(infos)])
    assert res[0] == res[1]


def test_instance_too_large_for_a_cluster(lib, oracle_lib):
    # 40,000 nodes need more than 16 CTAs of 2048 nodes: the batch runs on the
    # streaming kernels and still equals the single solves
    ds = make_batch([("uniform", 40000, 51, 10), ("mixture", 2000, 52, 10)])
    compare(oracle_lib, ds, _clusters())
