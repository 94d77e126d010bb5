"""The finisher's first phase on the GPU (one warp per block of 2,048 nodes)
against the same phase on the host threads: the same searches in the same
order, so whole solves agree bit for bit -- counters, augmentations, lambda,
x and the candidate graph -- for single instances, batches and degree
requirements, and an infeasible graph is reported alike."""
import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from paper_2011_08170_gb300 import build as B

pytestmark = pytest.mark.gpu

HOST, GPU = f2m.F2M_FLAG_FINISHER_HOST, f2m.F2M_FLAG_FINISHER_GPU
KEYS = ("status", "iterations", "phases", "pricing_rounds", "edges_added", "finisher_calls", "augmentations",
        "bound2", "frac_bits", "certified", "nnz")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


@pytest.mark.parametrize("kind,n,seed,k,cap", [("uniform", 30000, 0, 10, 256), ("mixture", 20000, 1, 8, 64),
                                               ("uniform", 9000, 2, 6, 1000000), ("mixture", 3000, 3, 10, 7)])
def test_gpu_phase1_equals_host_phase1(lib, kind, n, seed, k, cap):
    d = I.make_instance(kind, n, seed, k)
    out = {}
    for fl in (HOST, GPU):
        s = f2m.solve(d["xy"], d["row_ptr"], d["col"], params=f2m.f2m_default_params(flags=fl, max_iters=cap))
        out[fl] = s
        assert s.info["finish_phase1_gpu"] == (1 if fl == GPU and s.info["finisher_calls"] else 0)
    a, b = out[HOST], out[GPU]
    assert a.info["finisher_calls"] >= 1
    for key in KEYS:
        assert a.info[key] == b.info[key], key
    assert a.info["finish_aug_phase"] == b.info["finish_aug_phase"]
    assert np.array_equal(a.lam, b.lam) and np.array_equal(a.x2, b.x2) and np.array_equal(a.col, b.col)


def test_gpu_phase1_with_degree_requirements(lib):
    d = I.make_instance("uniform", 12000, 4, 10)
    rng = np.random.default_rng(5)
    b = np.minimum(rng.integers(1, 5, size=12000), np.diff(d["row_ptr"]) - 1).astype(np.int32)
    out = [f2m.solve(d["xy"], d["row_ptr"], d["col"], b=b, params=f2m.f2m_default_params(flags=fl))
           for fl in (HOST, GPU)]
    for key in KEYS:
        assert out[0].info[key] == out[1].info[key], key
    assert np.array_equal(out[0].lam, out[1].lam) and np.array_equal(out[0].x2, out[1].x2)


def test_gpu_phase1_in_batches(lib):
    rng = np.random.default_rng(11)
    specs = [("uniform" if i % 2 == 0 else "mixture", int(rng.integers(800, 6000)), 40 + i, 10) for i in range(20)]
    ds = [I.make_instance(*sp) for sp in specs]
    insts = [(d["xy"], d["row_ptr"], d["col"]) for d in ds]
    res = {}
    for fl in (HOST, GPU):
        bt = f2m.f2m_create_batch(insts, f2m.f2m_default_params(flags=fl))
        infos, tot = f2m.f2m_solve_batch(bt)
        res[fl] = (tot, [f2m.f2m_batch_get_lambda(bt, i) for i in range(len(ds))],
                   [f2m.f2m_batch_get_x(bt, i) for i in range(len(ds))])
        assert tot.status == 0 and tot.certified == 2
    (ta, la, xa), (tb, lb, xb) = res[HOST], res[GPU]
    assert ta.augmentations == tb.augmentations and ta.finish_phase1_gpu == 0 and tb.finish_phase1_gpu == 1
    for i in range(len(ds)):
        assert la[i][1] == lb[i][1] and np.array_equal(la[i][0], lb[i][0])
        for u, v in zip(xa[i], xb[i]):
            assert np.array_equal(u, v)


def test_gpu_phase1_infeasible_graph(lib):
    # K_{3,5}: the left side cannot supply what the right side needs
    xy = np.array([[0, 0], [0, 10], [0, 20]] + [[100, 7 * i] for i in range(5)], dtype=np.int32)
    rows = [[3, 4, 5, 6, 7]] * 3 + [[0, 1, 2]] * 5
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    for fl in (HOST, GPU):
        ctx = f2m.f2m_create(xy, rp, col, f2m.f2m_default_params(pricing=0, max_iters=2000, flags=fl))
        info = f2m.f2m_solve(ctx, raise_on_error=False)
        assert info.status in (f2m.F2M_ERR_INFEASIBLE, f2m.F2M_ERR_OVERFLOW)
