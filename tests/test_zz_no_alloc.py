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
    st = f2m.load().f2m_gdp_noalloc(rp.data_ptr(), ec.data_ptr(), 1000, 8, 2, 10, lam_h.ctypes.data,
                                    C.byref(sw), None, None, buf, 256)
    assert st == f2m.F2M_ERR_INVALID_ARG and b"device memory" in buf.value
