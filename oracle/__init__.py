"""ctypes wrapper of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  The CUDA library never loads it.

The oracle is plain single-threaded C (``f2m_oracle.c``, ``certify.c``), built
with ``gcc -O2`` and no fast-math by ``build()``.  Arrays cross as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["f2m_oracle.c", "certify.c", "subtour.c"]

OR_OK = 0
OR_INVALID = 1
OR_NOT_CONVERGED = 4
OR_OVERFLOW = 5
OR_PRICING_OVERFLOW = 6
OR_INFEASIBLE = 7


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES + ["f2m_oracle.h"]]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-fno-fast-math", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


class _Params(C.Structure):
    _fields_ = [("frac_bits", C.c_int32), ("damping_shift", C.c_int32),
                ("max_iters", C.c_int64), ("max_pricing_rounds", C.c_int32),
                ("pricing", C.c_int32), ("finisher", C.c_int32), ("update", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("phases", C.c_int64),
                ("pricing_rounds", C.c_int64), ("edges_added", C.c_int64),
                ("finisher_calls", C.c_int64), ("augmentations", C.c_int64),
                ("bound2", C.c_int64), ("frac_bits", C.c_int32),
                ("certified", C.c_int32), ("status", C.c_int32)]


class _SubtourInfo(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("phases", C.c_int64), ("pricing_rounds", C.c_int64),
                ("edges_added", C.c_int64), ("cuts", C.c_int64), ("bound2_f2m", C.c_int64),
                ("bound2", C.c_int64), ("rounds", C.c_int32), ("layers", C.c_int32),
                ("frac_bits", C.c_int32), ("certified", C.c_int32), ("status", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.or_nint_sqrt.restype = C.c_int64
        L.or_nint_sqrt.argtypes = [C.c_int64]
        L.or_nint_sqrt_array.argtypes = [C.c_int64, _i64p, _i64p]
        L.or_cost_table.argtypes = [C.c_int32, _i32p, _i32p, _i32p, _i32p]
        L.or_sweep.restype = C.c_int
        L.or_sweep.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, _i32p, C.c_int32, C.c_int32,
                               _i32p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.or_bound2.restype = C.c_int64
        L.or_bound2.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, _i32p, C.c_int32]
        L.or_gdp.restype = C.c_int
        L.or_gdp.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, C.c_int32, C.c_int32, C.c_int64,
                             _i32p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_int64]
        L.or_extract.restype = C.c_int64
        L.or_extract.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, _i32p, C.c_int32, _u8p]
        L.or_finisher.restype = C.c_int
        L.or_finisher.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, _i32p, C.c_int32, _u8p,
                                  _i32p, C.POINTER(C.c_int64)]
        L.or_pricing_rows.restype = C.c_int64
        L.or_pricing_rows.argtypes = [C.c_int32, _i32p, _i32p, _i32p, _i32p, C.c_int32,
                                      C.c_int32, C.c_int32, C.c_void_p, C.c_int64]
        L.or_merge.restype = C.c_int64
        L.or_merge.argtypes = [C.c_int32, _i32p, _i32p, C.c_int64, _i32p, _i32p, _i32p]
        L.or_solve.restype = C.c_void_p
        L.or_solve.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, C.c_void_p,
                               C.POINTER(_Params), C.POINTER(_Info), C.c_void_p, C.c_void_p,
                               C.c_int64]
        L.or_result_nnz.restype = C.c_int64
        L.or_result_nnz.argtypes = [C.c_void_p]
        L.or_result_copy.argtypes = [C.c_void_p, _i32p, _i32p, _u8p, _i32p]
        L.or_result_free.argtypes = [C.c_void_p]
        L.or_certify.restype = C.c_int
        L.or_certify.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, _u8p, _i32p, C.c_int32,
                                 C.c_int64, C.c_int32]
        L.or_knn.argtypes = [C.c_int32, _i32p, C.c_int32, _i32p, _i64p]
        L.or_splitmix64.restype = C.c_uint64
        L.or_splitmix64.argtypes = [C.c_uint64]
        L.or_color_greedy.restype = C.c_int32
        L.or_color_greedy.argtypes = [C.c_int32, _i32p, _i32p, _i32p]
        L.or_gs_sweep.restype = C.c_int
        L.or_gs_sweep.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, _i32p, C.c_int32,
                                  _i32p, C.c_int32, C.c_int32, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]
        L.or_gdp_gs.restype = C.c_int
        L.or_gdp_gs.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, _i32p, C.c_int32,
                                C.c_int32, C.c_int32, C.c_int64, _i32p, C.POINTER(C.c_int64),
                                C.c_void_p, C.c_void_p, C.c_int64]
        L.or_cut_z.restype = C.c_int64
        L.or_cut_z.argtypes = [C.c_int32, _i32p, C.c_int32, C.c_void_p, C.c_void_p, _i32p, C.c_void_p,
                               C.c_int32, C.c_int32, C.c_int32]
        L.or_cut_bound2.restype = C.c_int64
        L.or_cut_bound2.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_int32, C.c_void_p, C.c_void_p,
                                    _i32p, C.c_void_p, C.c_int32]
        L.or_cut_sweep.restype = C.c_int
        L.or_cut_sweep.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_int32, C.c_void_p, C.c_void_p,
                                   _i32p, C.c_void_p, C.c_int32, C.c_int32, _i32p, C.c_void_p,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.or_cut_gdp.restype = C.c_int
        L.or_cut_gdp.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_int32, C.c_int32, C.c_int64, _i32p, C.c_void_p,
                                 C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_int64]
        L.or_cut_extract.restype = C.c_int64
        L.or_cut_extract.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_int32, C.c_void_p, C.c_void_p,
                                     _i32p, C.c_void_p, C.c_int32, _u8p]
        L.or_separate.restype = C.c_int32
        L.or_separate.argtypes = [C.c_int32, _i32p, _i32p, _u8p, _i32p]
        L.or_cut_pricing.restype = C.c_int64
        L.or_cut_pricing.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_int32, C.c_void_p, C.c_void_p,
                                     _i32p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int64]
        L.or_solve_subtour.restype = C.c_void_p
        L.or_solve_subtour.argtypes = [C.c_int32, _i32p, _i32p, _i32p, C.c_void_p, C.c_int32, C.c_int32,
                                       C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.POINTER(_SubtourInfo)]
        L.or_subtour_nnz.restype = C.c_int64
        L.or_subtour_nnz.argtypes = [C.c_void_p]
        L.or_subtour_cuts.restype = C.c_int64
        L.or_subtour_cuts.argtypes = [C.c_void_p]
        L.or_subtour_layers.restype = C.c_int32
        L.or_subtour_layers.argtypes = [C.c_void_p]
        L.or_subtour_copy.argtypes = [C.c_void_p] + [C.c_void_p] * 7
        L.or_subtour_free.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _degrees(b, n):
    """Degree requirements b_v as a contiguous int32 array, or None for b_v = 2
    (the fractional 2-matching).  A scalar b means b_v = b for every node."""
    if b is None:
        return None
    b = np.asarray(b)
    if b.ndim == 0:
        b = np.full(n, int(b), dtype=np.int32)
    b = _i32(b)
    if b.size != n:
        raise ValueError("b must hold one degree requirement per node")
    return b


def _ptr(a):
    return None if a is None else a.ctypes.data


def nint_sqrt(d2) -> np.ndarray:
    d2 = np.ascontiguousarray(d2, dtype=np.int64)
    out = np.empty_like(d2)
    lib().or_nint_sqrt_array(d2.size, d2.reshape(-1), out.reshape(-1))
    return out


def cost_table(xy, row_ptr, col) -> np.ndarray:
    xy, row_ptr, col = _i32(xy), _i32(row_ptr), _i32(col)
    out = np.empty(col.size, dtype=np.int32)
    lib().or_cost_table(row_ptr.size - 1, xy.reshape(-1), row_ptr, col, out)
    return out


def sweep(row_ptr, col, cost, lam, F=8, shift=2, b=None):
    """One Jacobi GDP sweep: returns (status, lam_new, bound2, changed).
    b: degree requirements (None: 2 everywhere; see or_sweep)."""
    row_ptr, col, cost, lam = _i32(row_ptr), _i32(col), _i32(cost), _i32(lam)
    bb = _degrees(b, lam.size)
    out = np.empty_like(lam)
    b2, ch = C.c_int64(), C.c_int64()
    st = lib().or_sweep(lam.size, row_ptr, col, cost, _ptr(bb), lam, F, shift, out, C.byref(b2),
                        C.byref(ch))
    return st, out, b2.value, ch.value


def bound2(row_ptr, col, cost, lam, fb=8, b=None) -> int:
    n = row_ptr.size - 1
    bb = _degrees(b, n)
    return int(lib().or_bound2(n, _i32(row_ptr), _i32(col), _i32(cost), _ptr(bb), _i32(lam), fb))


def gdp(row_ptr, col, cost, lam0, F=8, shift=2, max_iters=100000, trace=False, b=None):
    """GDP phase: returns (status, lam, iters, trace_bound2, trace_changed)."""
    lam = _i32(lam0).copy()
    bb = _degrees(b, lam.size)
    it = C.c_int64()
    tb = np.zeros(max_iters if trace else 1, dtype=np.int64)
    tc = np.zeros_like(tb)
    st = lib().or_gdp(lam.size, _i32(row_ptr), _i32(col), _i32(cost), _ptr(bb), F, shift, max_iters, lam,
                      C.byref(it), tb.ctypes.data if trace else None,
                      tc.ctypes.data if trace else None, max_iters if trace else 0)
    k = it.value
    return st, lam, k, (tb[:k] if trace else None), (tc[:k] if trace else None)


def splitmix64(seed: int) -> int:
    return int(lib().or_splitmix64(seed))


def color_greedy(row_ptr, col):
    """Greedy colouring in (degree, splitmix64, id) priority: (ncolors, color int32 [n])."""
    row_ptr, col = _i32(row_ptr), _i32(col)
    color = np.zeros(row_ptr.size - 1, dtype=np.int32)
    nc = lib().or_color_greedy(row_ptr.size - 1, row_ptr, col, color)
    return int(nc), color


def gs_sweep(row_ptr, col, cost, lam, color, ncolors, F=8, shift=1, b=None):
    """One class-by-class sweep: returns (status, lam_new, bound2 at the input, changed)."""
    row_ptr, col, cost = _i32(row_ptr), _i32(col), _i32(cost)
    out = _i32(lam).copy()
    bb = _degrees(b, out.size)
    b2, ch = C.c_int64(), C.c_int64()
    st = lib().or_gs_sweep(out.size, row_ptr, col, cost, _ptr(bb), _i32(color), ncolors, out, F,
                           shift, C.byref(b2), C.byref(ch))
    return st, out, b2.value, ch.value


def gdp_gs(row_ptr, col, cost, lam0, color, ncolors, F=8, shift=1, max_iters=100000, trace=False,
           b=None):
    """Class-by-class GDP phase: returns (status, lam, iters, trace_bound2, trace_changed)."""
    lam = _i32(lam0).copy()
    bb = _degrees(b, lam.size)
    it = C.c_int64()
    tb = np.zeros(max_iters if trace else 1, dtype=np.int64)
    tc = np.zeros_like(tb)
    st = lib().or_gdp_gs(lam.size, _i32(row_ptr), _i32(col), _i32(cost), _ptr(bb), _i32(color),
                         ncolors, F, shift, max_iters, lam, C.byref(it),
                         tb.ctypes.data if trace else None, tc.ctypes.data if trace else None,
                         max_iters if trace else 0)
    k = it.value
    return st, lam, k, (tb[:k] if trace else None), (tc[:k] if trace else None)


def extract(row_ptr, col, cost, lam, fb=8, b=None):
    n = row_ptr.size - 1
    bb = _degrees(b, n)
    x2 = np.zeros(np.asarray(col).size, dtype=np.uint8)
    bad = lib().or_extract(n, _i32(row_ptr), _i32(col), _i32(cost), _ptr(bb), _i32(lam), fb, x2)
    return int(bad), x2


def finisher(row_ptr, col, cost, lam, F=8, b=None):
    """Exact min-cost-flow finisher (plain successive shortest paths): returns
    (status, x2, lam2 at F+1 bits, augmentations)."""
    x2 = np.zeros(np.asarray(col).size, dtype=np.uint8)
    lam = _i32(lam)
    bb = _degrees(b, lam.size)
    lam2 = np.zeros_like(lam)
    aug = C.c_int64()
    st = lib().or_finisher(lam.size, _i32(row_ptr), _i32(col), _i32(cost),
                           _ptr(bb), lam, F, x2, lam2, C.byref(aug))
    return st, x2, lam2, aug.value


def pricing(xy, row_ptr, col, lam, fb=8, rows=None, cap=None):
    """Pairs (u < v) outside the CSR with negative reduced cost, ascending; int32 [m, 2]."""
    xy, row_ptr, col, lam = _i32(xy), _i32(row_ptr), _i32(col), _i32(lam)
    n = lam.size
    u0, u1 = (0, n) if rows is None else rows
    cnt = lib().or_pricing_rows(n, xy.reshape(-1), row_ptr, col, lam, fb, u0, u1, None, 0)
    if cap is not None and cnt > cap:
        return cnt, None
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    lib().or_pricing_rows(n, xy.reshape(-1), row_ptr, col, lam, fb, u0, u1, out.ctypes.data, cnt)
    return cnt, out[:cnt]


def merge(row_ptr, col, pairs):
    row_ptr, col = _i32(row_ptr), _i32(col)
    pairs = _i32(np.asarray(pairs).reshape(-1, 2))
    n = row_ptr.size - 1
    nrp = np.zeros(n + 1, dtype=np.int32)
    ncl = np.zeros(col.size + 2 * pairs.shape[0] + 1, dtype=np.int32)
    nnz = lib().or_merge(n, row_ptr, col, pairs.shape[0], pairs.reshape(-1) if pairs.size else np.zeros(2, np.int32), nrp, ncl)
    return nrp, ncl[:nnz].copy()


@dataclass
class OracleResult:
    status: int
    iterations: int
    phases: int
    pricing_rounds: int
    edges_added: int
    finisher_calls: int
    augmentations: int
    bound2: int
    frac_bits: int
    certified: int
    row_ptr: np.ndarray
    col: np.ndarray
    x2: np.ndarray
    lam: np.ndarray
    trace_bound2: np.ndarray | None = None
    trace_changed: np.ndarray | None = None

    @property
    def opt(self) -> float:
        """The dual bound as a length: bound2 / (2 * 2^frac_bits)."""
        return self.bound2 / (2.0 * (1 << self.frac_bits))


def solve(xy, row_ptr, col, lam0=None, F=8, shift=2, max_iters=128, max_pricing_rounds=64,
          pricing=True, finisher=True, trace_cap=0, b=None, classes=False) -> OracleResult:
    """max_iters: sweeps per GDP phase (a phase also ends at a fixed point; the
    solve goes on from the lambda reached either way).  classes: class-by-class
    (Gauss-Seidel) sweeps instead of Jacobi."""
    xy, row_ptr, col = _i32(xy), _i32(row_ptr), _i32(col)
    n = row_ptr.size - 1
    bb = _degrees(b, n)
    p = _Params(F, shift, max_iters, max_pricing_rounds, int(pricing), int(finisher), int(classes))
    info = _Info()
    lam0a = None if lam0 is None else _i32(lam0)
    tb = np.zeros(max(trace_cap, 1), dtype=np.int64)
    tc = np.zeros_like(tb)
    h = lib().or_solve(n, xy.reshape(-1), row_ptr, col, _ptr(bb),
                       None if lam0a is None else lam0a.ctypes.data, C.byref(p), C.byref(info),
                       tb.ctypes.data if trace_cap else None,
                       tc.ctypes.data if trace_cap else None, trace_cap)
    try:
        nnz = lib().or_result_nnz(h)
        rp = np.zeros(n + 1, dtype=np.int32)
        cl = np.zeros(max(nnz, 1), dtype=np.int32)
        x2 = np.zeros(max(nnz, 1), dtype=np.uint8)
        lam = np.zeros(n, dtype=np.int32)
        lib().or_result_copy(h, rp, cl, x2, lam)
    finally:
        lib().or_result_free(h)
    k = min(info.iterations, trace_cap)
    return OracleResult(info.status, info.iterations, info.phases, info.pricing_rounds,
                        info.edges_added, info.finisher_calls, info.augmentations, info.bound2,
                        info.frac_bits, info.certified, rp, cl[:nnz], x2[:nnz], lam,
                        tb[:k] if trace_cap else None, tc[:k] if trace_cap else None)


def certify(xy, row_ptr, col, x2, lam, fb, bound2, full_scan=True, b=None) -> int:
    """0 if (x2, lam) is certified optimal (see certify.c), else the failed check number."""
    xy, row_ptr, col = _i32(xy), _i32(row_ptr), _i32(col)
    bb = _degrees(b, row_ptr.size - 1)
    return int(lib().or_certify(row_ptr.size - 1, xy.reshape(-1), row_ptr, col, _ptr(bb),
                                np.ascontiguousarray(x2, dtype=np.uint8), _i32(lam), fb,
                                int(bound2), int(full_scan)))


def knn(xy, k):
    """k nearest neighbours by exact int64 squared distance, ties by smaller index
    (brute force, f2m_oracle.c): (nbr int32 [n, k], d2 int64 [n, k])."""
    xy = _i32(xy)
    n = xy.shape[0]
    nbr = np.zeros(n * k, dtype=np.int32)
    d2 = np.zeros(n * k, dtype=np.int64)
    lib().or_knn(n, xy.reshape(-1), k, nbr, d2)
    return nbr.reshape(n, k), d2.reshape(n, k)


def knn_csr(xy, k):
    """Symmetrised k-nearest-neighbour candidate graph (Section 5.3): u ~ w when
    either lists the other; rows sorted by column.  (row_ptr int32, col int32)."""
    nbr, _ = knn(xy, k)
    n = nbr.shape[0]
    u = np.repeat(np.arange(n, dtype=np.int64), k)
    w = nbr.reshape(-1).astype(np.int64)
    pairs = np.unique(np.concatenate([u * n + w, w * n + u]))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(pairs // n, minlength=n), out=row_ptr[1:])
    return row_ptr.astype(np.int32), (pairs % n).astype(np.int32)


# ---- subtour-elimination cuts (subtour.c) ------------------------------------

class Cuts:
    """A layered cut family: comp int32 [L, n] (-1: no cut of the layer, else the
    cut's index in its layer) and ncuts [L]."""

    def __init__(self, n, layers=()):
        self.n = n
        self.comp = np.zeros((0, n), dtype=np.int32)
        self.ncuts = np.zeros(0, dtype=np.int32)
        for comp, m in layers:
            self.add(comp, m)

    def add(self, comp, m):
        comp = _i32(comp).reshape(1, self.n)
        self.comp = np.ascontiguousarray(np.concatenate([self.comp, comp]), dtype=np.int32)
        self.ncuts = np.ascontiguousarray(np.append(self.ncuts, int(m)), dtype=np.int32)

    @property
    def L(self):
        return int(self.ncuts.size)

    @property
    def total(self):
        return int(self.ncuts.sum())

    def args(self):
        return (self.L, self.comp.ctypes.data if self.L else None,
                self.ncuts.ctypes.data if self.L else None)


def _mu(mu, cuts):
    mu = np.zeros(cuts.total, np.int32) if mu is None else _i32(mu).copy()
    assert mu.size == cuts.total
    return mu


def _mu_ptr(mu):
    return mu.ctypes.data if mu.size else None


def cut_z(xy, cuts, lam, mu, fb, u, v) -> int:
    mu = _mu(mu, cuts)
    return int(lib().or_cut_z(cuts.n, _i32(xy).reshape(-1), *cuts.args(), _i32(lam), _mu_ptr(mu), fb, u, v))


def cut_bound2(row_ptr, col, cost, cuts, lam, mu, fb=8) -> int:
    mu = _mu(mu, cuts)
    return int(lib().or_cut_bound2(cuts.n, _i32(row_ptr), _i32(col), _i32(cost), *cuts.args(), _i32(lam),
                                   _mu_ptr(mu), fb))


def cut_sweep(row_ptr, col, cost, cuts, lam, mu, F=8, shift=2):
    """One Jacobi sweep of node and cut duals: (status, lam, mu, bound2, changed)."""
    lam = _i32(lam)
    mu = _mu(mu, cuts)
    nl = np.zeros_like(lam)
    nm = np.zeros_like(mu)
    b2, ch = C.c_int64(), C.c_int64()
    st = lib().or_cut_sweep(cuts.n, _i32(row_ptr), _i32(col), _i32(cost), *cuts.args(), lam, _mu_ptr(mu),
                            F, shift, nl, _mu_ptr(nm), C.byref(b2), C.byref(ch))
    return st, nl, nm, b2.value, ch.value


def cut_gdp(row_ptr, col, cost, cuts, lam0, mu0=None, F=8, shift=2, max_iters=1000, trace=False):
    """GDP phase with cuts: (status, lam, mu, iters, trace_bound2, trace_changed)."""
    lam = _i32(lam0).copy()
    mu = _mu(mu0, cuts)
    it = C.c_int64()
    tb = np.zeros(max_iters if trace else 1, dtype=np.int64)
    tc = np.zeros_like(tb)
    st = lib().or_cut_gdp(cuts.n, _i32(row_ptr), _i32(col), _i32(cost), *cuts.args(), F, shift, max_iters,
                          lam, _mu_ptr(mu), C.byref(it), tb.ctypes.data if trace else None,
                          tc.ctypes.data if trace else None, max_iters if trace else 0)
    k = it.value
    return st, lam, mu, k, (tb[:k] if trace else None), (tc[:k] if trace else None)


def cut_extract(row_ptr, col, cost, cuts, lam, mu, fb=8):
    mu = _mu(mu, cuts)
    x2 = np.zeros(np.asarray(col).size, dtype=np.uint8)
    bad = lib().or_cut_extract(cuts.n, _i32(row_ptr), _i32(col), _i32(cost), *cuts.args(), _i32(lam),
                               _mu_ptr(mu), fb, x2)
    return int(bad), x2


def separate(row_ptr, col, x2):
    """One cut layer from the components of the support of x2: (comp [n], ncuts)."""
    n = np.asarray(row_ptr).size - 1
    comp = np.zeros(n, dtype=np.int32)
    m = lib().or_separate(n, _i32(row_ptr), _i32(col), np.ascontiguousarray(x2, dtype=np.uint8), comp)
    return comp, int(m)


def cut_pricing(xy, row_ptr, col, cuts, lam, mu, fb=8):
    """Pairs (u < v) outside the CSR with z < 0, cut duals included; int32 [m, 2]."""
    mu = _mu(mu, cuts)
    xy, row_ptr, col, lam = _i32(xy), _i32(row_ptr), _i32(col), _i32(lam)
    cnt = lib().or_cut_pricing(cuts.n, xy.reshape(-1), row_ptr, col, *cuts.args(), lam, _mu_ptr(mu), fb,
                               None, 0)
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    lib().or_cut_pricing(cuts.n, xy.reshape(-1), row_ptr, col, *cuts.args(), lam, _mu_ptr(mu), fb,
                         out.ctypes.data, cnt)
    return int(cnt), out[:cnt]


@dataclass
class SubtourResult:
    info: dict
    row_ptr: np.ndarray
    col: np.ndarray
    x2: np.ndarray
    lam: np.ndarray
    mu: np.ndarray
    cuts: "Cuts"


def solve_subtour(xy, row_ptr, col, rounds=3, lam0=None, F=8, shift=2, max_iters=128, pricing=True,
                  max_pricing_rounds=64) -> SubtourResult:
    """Stages of GDP with pricing and subtour-cut layers between them (subtour.c)."""
    xy, row_ptr, col = _i32(xy), _i32(row_ptr), _i32(col)
    n = row_ptr.size - 1
    info = _SubtourInfo()
    lam0a = None if lam0 is None else _i32(lam0)
    h = lib().or_solve_subtour(n, xy.reshape(-1), row_ptr, col, None if lam0a is None else lam0a.ctypes.data,
                               F, shift, max_iters, int(pricing), max_pricing_rounds, rounds, C.byref(info))
    try:
        nnz = lib().or_subtour_nnz(h)
        M = lib().or_subtour_cuts(h)
        L = lib().or_subtour_layers(h)
        rp = np.zeros(n + 1, np.int32)
        cl = np.zeros(max(nnz, 1), np.int32)
        x2 = np.zeros(max(nnz, 1), np.uint8)
        lam = np.zeros(n, np.int32)
        mu = np.zeros(max(M, 1), np.int32)
        comp = np.zeros((max(L, 1), n), np.int32)
        ncuts = np.zeros(max(L, 1), np.int32)
        lib().or_subtour_copy(h, rp.ctypes.data, cl.ctypes.data, x2.ctypes.data, lam.ctypes.data,
                              mu.ctypes.data, comp.ctypes.data, ncuts.ctypes.data)
    finally:
        lib().or_subtour_free(h)
    cuts = Cuts(n, [(comp[l], int(ncuts[l])) for l in range(L)])
    d = {k: getattr(info, k) for k, _ in _SubtourInfo._fields_}
    return SubtourResult(d, rp, cl[:nnz], x2[:nnz], lam, mu[:M], cuts)
