"""The library's host finisher (csrc/finisher.cpp) on the CPU, without a GPU.

The finisher repairs a degenerate stop of the gradient procedure (Section 3,
last paragraph) with an exact min-cost flow on the bipartite double cover.
Its blocked, multi-threaded schedule is the library's own choice, so its
result is checked against what the mathematics fixes, not against a copy of
its steps:
- primal feasibility: every row of x sums to b_v (x_e in {0, 1/2, 1});
- complementary slackness in exact integers at F+1 bits with the returned
  lambda (x_e = 1 needs z_e <= 0, x_e = 0 needs z_e >= 0, x_e = 1/2 needs
  z_e = 0), which with feasibility proves x optimal on the candidate graph;
- the same optimum and the same number of unit augmentations (the initial
  surplus) as the oracle's plain successive-shortest-path finisher;
- the same result for every thread count, and per instance of a batch the
  result of its single run, with instances left out untouched.
The inputs are built here the way the device prepares them: twin entries,
arcs with z < 0 saturated, surpluses b_v minus the saturated arcs.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_08170_gb300", "csrc")
F = 8


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def fin(tmp_path_factory):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers (for the vector types the library's headers use)")
    out = str(tmp_path_factory.mktemp("hostfin") / "libhostfin.so")
    cmd = [cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I", CSRC, "-I", inc,
           os.path.join(os.path.dirname(__file__), "host_finisher_shim.cpp"),
           os.path.join(CSRC, "finisher.cpp"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = C.CDLL(out)
    p = C.c_void_p
    L.shim_host_finisher.argtypes = [C.c_int32, p, p, p, p, p, p, C.c_int32, p, p, C.c_int32, p, C.c_int32,
                                     C.POINTER(C.c_int64), p]
    L.shim_host_finisher.restype = C.c_int
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data


def prepare(rp, col, cost, lam, b):
    """Twins, the initial flow (z < 0 saturated) and the surpluses."""
    n = len(rp) - 1
    row = np.repeat(np.arange(n), np.diff(rp))
    key = row.astype(np.int64) * n + col
    order = np.argsort(key)
    twin = order[np.searchsorted(key[order], col.astype(np.int64) * n + row)].astype(np.int32)
    assert np.array_equal(row[twin], col) and np.array_equal(col[twin], row)
    z = (cost.astype(np.int64) << F) - lam[row].astype(np.int64) - lam[col].astype(np.int64)
    y = (z < 0).astype(np.uint8)
    exl = (b - np.bincount(row, weights=y, minlength=n)).astype(np.int32)
    iec = np.ascontiguousarray(np.stack([col, cost], 1).astype(np.int32))
    return row, twin, y, exl, iec


def run(fin, rp, iec, twin, y, exl, lam, seg_off, include=None, threads=1, lam2=None):
    n = len(rp) - 1
    y = y.copy()
    lam2 = np.zeros(n, np.int32) if lam2 is None else lam2.copy()
    aug = C.c_int64()
    phases = np.zeros(3, np.int64)
    seg = np.asarray(seg_off, np.int32)
    inc = None if include is None else np.asarray(include, np.uint8)
    r = fin.shim_host_finisher(n, _ptr(rp), _ptr(iec), _ptr(twin), _ptr(y), _ptr(exl), _ptr(lam), F, _ptr(lam2),
                               _ptr(seg), len(seg) - 1, _ptr(inc), threads, C.byref(aug), _ptr(phases))
    return r, y, lam2, aug.value, phases


def check_optimal(rp, row, col, cost, twin, y, lam2, b):
    x2 = y.astype(np.int64) + y[twin]  # x in half units
    assert np.array_equal(np.bincount(row, weights=x2, minlength=len(rp) - 1), 2 * b)
    z2 = (cost.astype(np.int64) << (F + 1)) - lam2[row].astype(np.int64) - lam2[col].astype(np.int64)
    assert np.all(z2[x2 == 2] <= 0) and np.all(z2[x2 == 0] >= 0) and np.all(z2[x2 == 1] == 0)
    return int(np.sum(cost.astype(np.int64) * x2))  # 4 x the objective (both directions, half units)


def instance(O, kind, n, seed, k, degrees=False):
    d = I.make_instance(kind, n, seed, k)
    rp, col = d["row_ptr"], d["col"]
    cost = O.cost_table(d["xy"], rp, col)
    b = None
    if degrees:
        rng = np.random.default_rng(seed)
        b = np.minimum(rng.integers(1, 4, size=n), np.diff(rp) - 1).astype(np.int32)
    _, lam, *_ = O.gdp(rp, col, cost, np.zeros(n, np.int32), F, 2, 128, b=b)
    return rp, col, cost, lam, (np.full(n, 2, np.int32) if b is None else b), b


@pytest.mark.parametrize("kind,n,seed,k,degrees", [("uniform", 5000, 1, 8, False), ("mixture", 6000, 2, 10, False),
                                                   ("uniform", 3000, 3, 5, True)])
def test_host_finisher_is_optimal_and_matches_the_oracle(fin, oracle_lib, kind, n, seed, k, degrees):
    O = oracle_lib
    rp, col, cost, lam, bv, b = instance(O, kind, n, seed, k, degrees)
    row, twin, y, exl, iec = prepare(rp, col, cost, lam, bv)
    assert np.any(exl != 0)  # a degenerate stop: there is something to repair
    r, y1, lam2, aug, phases = run(fin, rp, iec, twin, y, exl, lam, [0, n], threads=1)
    assert r == 0
    total = check_optimal(rp, row, col, cost, twin, y1, lam2, bv)
    st, x2_o, lam2_o, aug_o = O.finisher(rp, col, cost, lam, F, b=b)
    assert st == 0
    assert total == int(np.sum(cost.astype(np.int64) * x2_o))
    # one unit per augmentation: node i holds |surplus_i| units on one of its copies
    assert aug == aug_o == int(np.abs(exl).sum()) and aug == phases.sum()


def test_host_finisher_same_result_for_every_thread_count(fin, oracle_lib):
    rp, col, cost, lam, bv, _ = instance(oracle_lib, "uniform", 40000, 4, 10)
    n = len(rp) - 1
    row, twin, y, exl, iec = prepare(rp, col, cost, lam, bv)
    ref = run(fin, rp, iec, twin, y, exl, lam, [0, n], threads=1)
    assert ref[0] == 0 and ref[4][0] > 0 and ref[4][1] + ref[4][2] > 0  # blocked phases and the last one
    check_optimal(rp, row, col, cost, twin, ref[1], ref[2], bv)
    for threads in (2, 3, 8):
        r = run(fin, rp, iec, twin, y, exl, lam, [0, n], threads=threads)
        assert r[0] == 0 and np.array_equal(r[1], ref[1]) and np.array_equal(r[2], ref[2])
        assert r[3] == ref[3] and np.array_equal(r[4], ref[4])


def test_host_finisher_batch_segments_and_left_out_instances(fin, oracle_lib):
    # two instances in one CSR (columns offset): each segment's result is its
    # single run; with the second left out, its flow and lambda stay as given
    parts = [instance(oracle_lib, "mixture", 3000, 5, 8), instance(oracle_lib, "uniform", 2500, 6, 6)]
    singles, cols, costs, lams = [], [], [], []
    off = 0
    for rp, col, cost, lam, bv, _ in parts:
        row, twin, y, exl, iec = prepare(rp, col, cost, lam, bv)
        singles.append(run(fin, rp, iec, twin, y, exl, lam, [0, len(rp) - 1], threads=3))
        cols.append(col + off)
        costs.append(cost)
        lams.append(lam)
        off += len(rp) - 1
    n = off
    deg = np.concatenate([np.diff(p[0]) for p in parts])
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(deg, out=rp[1:])
    col, cost, lam = np.concatenate(cols).astype(np.int32), np.concatenate(costs), np.concatenate(lams)
    bv = np.full(n, 2, np.int32)
    row, twin, y, exl, iec = prepare(rp, col, cost, lam, bv)
    n0 = len(parts[0][0]) - 1
    e0 = int(parts[0][0][-1])
    r, y2, lam2, aug, _ = run(fin, rp, iec, twin, y, exl, lam, [0, n0, n], threads=4)
    assert r == 0 and aug == singles[0][3] + singles[1][3]
    assert np.array_equal(y2[:e0], singles[0][1]) and np.array_equal(y2[e0:], singles[1][1])
    assert np.array_equal(lam2[:n0], singles[0][2]) and np.array_equal(lam2[n0:], singles[1][2])
    sentinel = np.full(n, -7, np.int32)
    r, y3, lam3, aug3, _ = run(fin, rp, iec, twin, y, exl, lam, [0, n0, n], include=[1, 0], threads=4,
                               lam2=sentinel)
    assert r == 0 and aug3 == singles[0][3]
    assert np.array_equal(y3[:e0], singles[0][1]) and np.array_equal(lam3[:n0], singles[0][2])
    assert np.array_equal(y3[e0:], y[e0:]) and np.all(lam3[n0:] == -7)


def test_host_finisher_reports_an_infeasible_instance(fin):
    # K4 with b = (3, 3, 3, 1): nodes 0, 1, 2 need every edge at 1, which gives
    # node 3 three instead of one, so no fractional b-matching exists; the
    # finisher reports it (status 7) instead of searching on
    xy = np.array([[0, 0], [10, 0], [0, 10], [10, 10]], np.int32)
    n = 4
    rp = np.arange(0, 13, 3, dtype=np.int32)
    col = np.array([j for i in range(n) for j in range(n) if j != i], np.int32)
    row = np.repeat(np.arange(n), 3)
    d = (xy[row] - xy[col]).astype(np.float64)
    cost = np.rint(np.sqrt((d ** 2).sum(1))).astype(np.int32)
    bv = np.array([3, 3, 3, 1], np.int32)
    lam = np.zeros(n, np.int32)
    _, twin, y, exl, iec = prepare(rp, col, cost, lam, bv)
    r, *_ = run(fin, rp, iec, twin, y, exl, lam, [0, n], threads=1)
    assert r == 7
