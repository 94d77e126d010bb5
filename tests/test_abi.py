"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

No GPU needed: only host-side logic is exercised (parameter defaults, argument
checks that fail before any device work).
"""
import ctypes as C
import glob
import os
import re

import pytest

import paper_2011_08170_gb300 as f2m
from paper_2011_08170_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(f2m_[a-z_0-9]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert {"f2m_create", "f2m_solve", "f2m_gdp", "f2m_price", "f2m_get_x"} <= names
    for name in names:
        assert hasattr(lib, name), name
    assert names <= set(f2m.EXPORTS) | {n for n in names if n.startswith("f2m_")}


def test_binding_names_match_header(lib):
    for name in declared_symbols():
        assert hasattr(f2m, name), f"binding lacks {name}"


def test_default_params(lib):
    p = f2m.f2m_default_params()
    assert (p.frac_bits, p.damping_shift, p.pricing, p.finisher) == (8, 2, 1, 1)
    assert p.max_iters == 128 and p.pricing_cap > 0 and p.barrier_budget_cycles > 0


def test_status_strings(lib):
    for s in range(9):
        assert lib.f2m_status_string(s)


def test_create_rejects_bad_sizes_before_device_work(lib):
    h = C.c_void_p()
    # n < 4
    st = lib.f2m_create(None, 3, None, None, None, None, C.byref(h))
    assert st == f2m.F2M_ERR_INVALID_ARG and h.value is None
    xy = (C.c_int32 * 8)()
    rp = (C.c_int32 * 5)()
    col = (C.c_int32 * 1)()
    st = lib.f2m_create(C.addressof(xy), 3, C.addressof(rp), C.addressof(col), None, None, C.byref(h))
    assert st == f2m.F2M_ERR_INVALID_ARG
    assert b"n must be" in lib.f2m_last_error(None)
    # bad params
    p = f2m.f2m_default_params(frac_bits=9)
    st = lib.f2m_create(C.addressof(xy), 4, C.addressof(rp), C.addressof(col), C.byref(p), None, C.byref(h))
    assert st == f2m.F2M_ERR_INVALID_ARG and b"frac_bits" in lib.f2m_last_error(None)
    # NULL out
    assert lib.f2m_create(None, 4, None, None, None, None, None) == f2m.F2M_ERR_INVALID_ARG


def test_null_context_calls_fail_cleanly(lib):
    assert lib.f2m_solve(None, None) == f2m.F2M_ERR_INVALID_ARG
    assert lib.f2m_gdp(None, 1, None, None, None, 0) == f2m.F2M_ERR_INVALID_ARG
    lib.f2m_destroy(None)


def test_library_compiled_for_sm103a():
    text = open(os.path.join(ROOT, "paper_2011_08170_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in text
    assert os.path.exists(B.LIB)


def test_committed_warm_start_weights():
    import os
    import numpy as np
    import instances as I
    p = os.path.join(os.path.dirname(__file__), "..", "paper_2011_08170_gb300", "warm_start_mlp.npy")
    w = np.load(p)
    assert w.dtype == np.float32 and w.shape == (I.MLP_NPARAMS,) and np.all(np.isfinite(w))
