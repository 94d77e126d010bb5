"""f2m_gdp_noalloc: the GDP phase for callers that cannot allocate device memory.

Its scratch lives in a fixed device array inside the library instead of memory
allocated per context.  It must give the same lambda, sweep count and bound as
the allocating entry point f2m_gdp, call after call, since every call reuses
(and must clear) the same array.  This file is collected last.
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


def device_inputs(d):
    import torch
    ctx = f2m.f2m_create(d["xy"], d["row_ptr"], d["col"])
    rp, col, _, cost = f2m.f2m_get_x(ctx)
    ec = np.stack([col, cost], axis=1).astype(np.int32)
    return ctx, torch.from_numpy(rp).cuda(), torch.from_numpy(np.ascontiguousarray(ec)).cuda()


@pytest.mark.parametrize("kind,n,seed,k", [("uniform", 5000, 0, 10), ("mixture", 3000, 2, 12)])
def test_matches_allocating_entry_point_two_calls_in_a_row(lib, kind, n, seed, k):
    import torch
    d = I.make_instance(kind, n, seed, k)
    ref, rp, ec = device_inputs(d)
    lam = torch.zeros(n, dtype=torch.int32, device="cuda")
    # call 1: a capped phase; call 2: continue in place to the fixed point
    for cap in (57, 10 ** 6):
        st_r, sw_r, tb, _ = f2m.f2m_gdp(ref, cap, trace_cap=cap if cap < 100 else 0)
        st, sw, b2, msg = f2m.f2m_gdp_noalloc(rp, ec, lam, cap)
        torch.cuda.synchronize()
        lam_r, _ = f2m.f2m_get_lambda(ref)
        assert st == st_r and sw == sw_r, msg
        assert np.array_equal(lam.cpu().numpy(), lam_r)
        if tb is not None:
            assert b2 == tb[-1]
    assert st == f2m.F2M_OK
    b_ref, _ = f2m.f2m_get_bound(ref)
    assert b2 == b_ref  # at a fixed point the last sweep's bound is the bound at lambda


def test_rejects_sizes_beyond_the_scratch_array(lib):
    import torch
    n = (1 << 18) + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ec = torch.zeros((3, 2), dtype=torch.int32, device="cuda")
    lam = torch.zeros(n, dtype=torch.int32, device="cuda")
    st, sw, _, msg = f2m.f2m_gdp_noalloc(rp, ec, lam, 10)
    assert st == f2m.F2M_ERR_INVALID_ARG and "262144" in msg


def test_rejects_host_lambda(lib):
    import ctypes as C
    import torch
    d = I.make_instance("uniform", 1000, 1, 10)
    ref, rp, ec = device_inputs(d)
    lam_h = np.zeros(1000, np.int32)
    sw = C.c_int64()
    buf = C.create_string_buffer(256)
    st = f2m.load().f2m_gdp_noalloc(rp.data_ptr(), ec.data_ptr(), int(ec.shape[0]), 1000, 8, 2, 10,
                                    lam_h.ctypes.data, C.byref(sw), None, None, buf, 256)
    assert st == f2m.F2M_ERR_INVALID_ARG and b"device memory" in buf.value


def _k37():
    # K_{3,7}: no fractional 2-matching exists, so GDP raises lambda without
    # bound and overflows after 6,607,470 sweeps from lambda = 0
    m = 7
    xy = np.array([[0, 0], [0, 10], [0, 20]] + [[100, 7 * i] for i in range(m)], dtype=np.int32)
    rows = [list(range(3, 3 + m))] * 3 + [[0, 1, 2]] * m
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate(rows).astype(np.int32)
    return {"xy": xy, "row_ptr": rp, "col": col}


def test_overflow_on_either_parity_of_the_last_sweep(lib, oracle_lib):
    # started 11 and 10 sweeps before the overflow (states from the oracle's
    # run from lambda = 0), the overflowing sweep is odd and even: status,
    # sweep count, lambda (left at the overflowing sweep's input, in whichever
    # half of the double buffer that is) and bound as the allocating entry point
    import torch
    d = _k37()
    O = oracle_lib
    cost = O.cost_table(d["xy"], d["row_ptr"], d["col"])
    z = np.zeros(10, np.int32)
    st_a, lam_a, _, _, _ = O.gdp(d["row_ptr"], d["col"], cost, z, 8, 2, 6607470 - 11)
    st_b, lam_b, _, _, _ = O.gdp(d["row_ptr"], d["col"], cost, lam_a, 8, 2, 1)
    assert st_a == st_b == O.OR_NOT_CONVERGED
    ref, rp, ec = device_inputs(d)
    for start, back in ((lam_a, 11), (lam_b, 10)):
        f2m.f2m_set_lambda(ref, start, 8)
        st_r, sw_r, tb, _ = f2m.f2m_gdp(ref, 50, trace_cap=50)
        lam_r, _ = f2m.f2m_get_lambda(ref)
        lam = torch.from_numpy(start.copy()).cuda()
        st, sw, b2, msg = f2m.f2m_gdp_noalloc(rp, ec, lam, 50)
        assert st == st_r == f2m.F2M_ERR_OVERFLOW and sw == sw_r == back, (st, sw, msg)
        assert np.array_equal(lam.cpu().numpy(), lam_r)
        assert b2 == tb[sw - 1]


def test_rejects_invalid_inputs_without_reading_out_of_bounds(lib):
    # each array is of the size the arguments state; only its contents are
    # wrong, so the check kernel's reads stay inside them
    import torch
    d = I.make_instance("uniform", 2000, 3, 10)
    ref, rp, ec = device_inputs(d)
    n = 2000
    lam = torch.zeros(n, dtype=torch.int32, device="cuda")
    cases = []
    e1 = ec.clone(); e1[int(rp[700]), 0] = n + 5; cases.append((rp, e1, lam, "column outside"))
    e2 = ec.clone(); e2[int(rp[701]), 0] = -1; cases.append((rp, e2, lam, "column outside"))
    e3 = ec.clone(); e3[int(rp[702]) + 1, 0] = 702; cases.append((rp, e3, lam, "self-loop"))
    e4 = ec.clone(); e4[int(rp[703]), 1] = 1 << 21; cases.append((rp, e4, lam, "cost"))
    r5 = rp.clone(); r5[900] = r5[902]; cases.append((r5, ec, lam, "row_ptr"))
    r6 = rp.clone(); r6[n] -= 1; cases.append((r6, ec, lam, "row_ptr"))
    l7 = lam.clone(); l7[55] = 1 << 29; cases.append((rp, ec, l7, "lambda"))
    for r, e, l, word in cases:
        before = l.clone()
        st, sw, _, msg = f2m.f2m_gdp_noalloc(r, e, l, 10)
        assert st == f2m.F2M_ERR_INVALID_ARG and word in msg, (word, st, msg)
        assert torch.equal(l, before)
    # the shared array was left dirty by the refused calls: a valid call after
    # them still equals the allocating entry point
    st_r, sw_r, *_ = f2m.f2m_gdp(ref, 40)
    st, sw, _, msg = f2m.f2m_gdp_noalloc(rp, ec, lam, 40)
    assert st == st_r and sw == sw_r == 40, msg
    assert np.array_equal(lam.cpu().numpy(), f2m.f2m_get_lambda(ref)[0])
