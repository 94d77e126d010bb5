"""Python binding of the f2m C ABI (include/f2m.h): argument marshalling only.

Every step of the solve runs in the CUDA library ``_build/libf2m.so`` (built by
``paper_2011_08170_gb300.build.build()``).  There is no fallback: if the library
is missing or no GPU is present, ``load()`` raises.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); outputs are
numpy arrays unless ``device`` is given, in which case they are torch tensors
allocated there.  Work runs on ``torch.cuda.current_stream()`` unless a stream
is passed to ``f2m_create``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libf2m.so")

F2M_OK = 0
F2M_ERR_INVALID_ARG = 1
F2M_ERR_CUDA = 2
F2M_ERR_OOM = 3
F2M_ERR_NOT_CONVERGED = 4
F2M_ERR_OVERFLOW = 5
F2M_ERR_PRICING_OVERFLOW = 6
F2M_ERR_INFEASIBLE = 7
F2M_ERR_TIMEOUT = 8

F2M_FLAG_STREAMING_GDP = 1
F2M_FLAG_ONE_SWEEP_GDP = 2
F2M_FLAG_CLASS_SWEEPS = 4
F2M_FLAG_BATCH_CLUSTERS = 8
F2M_FLAG_FINISHER_HOST = 16
F2M_FLAG_FINISHER_GPU = 32
F2M_FLAG_PRICING_TENSOR = 64
F2M_GDP_KERNEL_STREAMING, F2M_GDP_KERNEL_TILED, F2M_GDP_KERNEL_TWO_SWEEP = 0, 1, 2
F2M_GDP_KERNEL_TWO_SWEEP_PACKED, F2M_GDP_KERNEL_CLASSES = 3, 4
F2M_GDP_KERNEL_BATCH, F2M_GDP_KERNEL_BATCH_CLUSTERS = 5, 6

# every symbol the header declares
EXPORTS = ["f2m_default_params", "f2m_create", "f2m_destroy", "f2m_set_lambda", "f2m_solve",
           "f2m_gdp", "f2m_price", "f2m_add_edges", "f2m_extract", "f2m_get_lambda",
           "f2m_get_bound", "f2m_get_x", "f2m_status_string", "f2m_last_error",
           "f2m_kernel_launches", "f2m_gdp_noalloc", "f2m_create_batch", "f2m_solve_batch",
           "f2m_batch_get_lambda", "f2m_batch_get_x", "f2m_batch_last_error", "f2m_destroy_batch",
           "f2m_knn", "f2m_knn_csr", "f2m_features", "f2m_mlp_create", "f2m_mlp_destroy",
           "f2m_mlp_get_params", "f2m_mlp_last_error", "f2m_mlp_forward", "f2m_mlp_grad",
           "f2m_mlp_train", "f2m_warm_start", "f2m_set_degrees", "f2m_get_colors",
           "f2m_tsplib_parse", "f2m_tsplib_last_error", "f2m_separate", "f2m_add_cut_layer",
           "f2m_get_cut_duals", "f2m_solve_subtour", "f2m_pricing_mma_check"]

F2M_MLP_NPARAMS = 18817


class f2m_params(C.Structure):
    _fields_ = [("frac_bits", C.c_int32), ("damping_shift", C.c_int32),
                ("max_iters", C.c_int64), ("max_pricing_rounds", C.c_int32),
                ("pricing", C.c_int32), ("pricing_cap", C.c_int64),
                ("barrier_budget_cycles", C.c_int64), ("finisher", C.c_int32),
                ("flags", C.c_uint32), ("gdp_lanes", C.c_int32), ("gdp_ctas_per_sm", C.c_int32),
                ("batch_shape", C.c_int32), ("batch_graph", C.c_int32)]


class f2m_train_params(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float),
                ("lr_final_frac", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("seed", C.c_uint64)]


class f2m_info(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("phases", C.c_int64),
                ("pricing_rounds", C.c_int64), ("edges_added", C.c_int64),
                ("finisher_calls", C.c_int64), ("augmentations", C.c_int64),
                ("bound2", C.c_int64), ("nnz", C.c_int64), ("frac_bits", C.c_int32),
                ("certified", C.c_int32), ("status", C.c_int32), ("batch_shape", C.c_int32),
                ("batch_graph", C.c_int32), ("gdp_kernel", C.c_int32),
                ("ms_gdp", C.c_double), ("ms_pricing", C.c_double), ("ms_merge", C.c_double),
                ("ms_extract", C.c_double), ("ms_finish", C.c_double), ("ms_total", C.c_double),
                ("ms_finish_prep", C.c_double), ("ms_finish_phase", C.c_double * 3),
                ("ms_finish_scatter", C.c_double), ("finish_aug_phase", C.c_int64 * 3),
                ("finish_threads", C.c_int32), ("finish_phase1_gpu", C.c_int32),
                ("pricing_pairs", C.c_int64), ("certifying_scans", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self) -> dict:
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


class f2m_subtour_info(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("phases", C.c_int64), ("pricing_rounds", C.c_int64),
                ("edges_added", C.c_int64), ("cuts", C.c_int64), ("bound2_f2m", C.c_int64),
                ("bound2", C.c_int64), ("rounds", C.c_int32), ("layers", C.c_int32),
                ("frac_bits", C.c_int32), ("certified", C.c_int32), ("status", C.c_int32),
                ("pad", C.c_int32), ("ms_gdp", C.c_double), ("ms_pricing", C.c_double),
                ("ms_merge", C.c_double), ("ms_separate", C.c_double), ("ms_total", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class F2MError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libf2m.so and declare its signatures.  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"the f2m CUDA library is not built ({path}); run "
                           "paper_2011_08170_gb300.build.build() first")
    L = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.f2m_default_params.argtypes = [C.POINTER(f2m_params)]
    L.f2m_default_params.restype = None
    L.f2m_create.argtypes = [vp, i32, vp, vp, C.POINTER(f2m_params), vp, C.POINTER(vp)]
    L.f2m_destroy.argtypes = [vp]
    L.f2m_destroy.restype = None
    L.f2m_set_lambda.argtypes = [vp, vp, i32]
    L.f2m_set_degrees.argtypes = [vp, vp]
    L.f2m_get_colors.argtypes = [vp, vp, C.POINTER(i32)]
    L.f2m_tsplib_parse.argtypes = [C.c_char_p, i64, vp, i32, C.POINTER(i32), vp]
    L.f2m_tsplib_parse.restype = C.c_int
    L.f2m_tsplib_last_error.argtypes = []
    L.f2m_tsplib_last_error.restype = C.c_char_p
    L.f2m_solve.argtypes = [vp, C.POINTER(f2m_info)]
    L.f2m_gdp.argtypes = [vp, i64, C.POINTER(i64), vp, vp, i64]
    L.f2m_price.argtypes = [vp, C.POINTER(i64), vp, i64]
    L.f2m_add_edges.argtypes = [vp, vp, i64]
    L.f2m_extract.argtypes = [vp, vp, C.POINTER(i64)]
    L.f2m_get_lambda.argtypes = [vp, vp, C.POINTER(i32)]
    L.f2m_get_bound.argtypes = [vp, C.POINTER(i64), C.POINTER(i32)]
    L.f2m_get_x.argtypes = [vp, C.POINTER(i64), vp, vp, vp, vp]
    L.f2m_status_string.argtypes = [i32]
    L.f2m_status_string.restype = C.c_char_p
    L.f2m_last_error.argtypes = [vp]
    L.f2m_last_error.restype = C.c_char_p
    L.f2m_gdp_noalloc.argtypes = [vp, vp, i64, i32, i32, i32, i64, vp, C.POINTER(i64),
                                  C.POINTER(i64), vp, C.c_char_p, i64]
    L.f2m_gdp_noalloc.restype = C.c_int
    L.f2m_create_batch.argtypes = [i32, vp, vp, vp, vp, C.POINTER(f2m_params), vp, C.POINTER(vp)]
    L.f2m_create_batch.restype = C.c_int
    L.f2m_solve_batch.argtypes = [vp, vp, C.POINTER(f2m_info)]
    L.f2m_solve_batch.restype = C.c_int
    L.f2m_batch_get_lambda.argtypes = [vp, i32, vp, C.POINTER(i32)]
    L.f2m_batch_get_lambda.restype = C.c_int
    L.f2m_batch_get_x.argtypes = [vp, i32, C.POINTER(i64), vp, vp, vp]
    L.f2m_batch_get_x.restype = C.c_int
    L.f2m_batch_last_error.argtypes = [vp]
    L.f2m_batch_last_error.restype = C.c_char_p
    L.f2m_destroy_batch.argtypes = [vp]
    L.f2m_destroy_batch.restype = None
    L.f2m_knn.argtypes = [vp, i32, i32, vp, vp, vp]
    L.f2m_knn_csr.argtypes = [vp, i32, i32, vp, vp, C.POINTER(i64), vp]
    L.f2m_features.argtypes = [vp, i32, vp, vp, vp]
    L.f2m_mlp_create.argtypes = [vp, vp, C.POINTER(vp)]
    L.f2m_mlp_destroy.argtypes = [vp]
    L.f2m_mlp_destroy.restype = None
    L.f2m_mlp_get_params.argtypes = [vp, vp]
    L.f2m_mlp_last_error.argtypes = [vp]
    L.f2m_mlp_last_error.restype = C.c_char_p
    L.f2m_mlp_forward.argtypes = [vp, vp, i64, vp]
    L.f2m_mlp_grad.argtypes = [vp, vp, vp, i64, vp, vp]
    L.f2m_mlp_train.argtypes = [vp, vp, vp, i64, C.POINTER(f2m_train_params), vp]
    L.f2m_warm_start.argtypes = [vp, vp, C.POINTER(C.c_double)]
    for name in ("f2m_knn", "f2m_knn_csr", "f2m_features", "f2m_mlp_create", "f2m_mlp_get_params",
                 "f2m_mlp_forward", "f2m_mlp_grad", "f2m_mlp_train", "f2m_warm_start"):
        getattr(L, name).restype = C.c_int
    L.f2m_separate.argtypes = [vp, vp, C.POINTER(i32)]
    L.f2m_add_cut_layer.argtypes = [vp, vp, i32]
    L.f2m_get_cut_duals.argtypes = [vp, vp, C.POINTER(i64), C.POINTER(i32)]
    L.f2m_solve_subtour.argtypes = [vp, i32, C.POINTER(f2m_subtour_info)]
    for name in ("f2m_separate", "f2m_add_cut_layer", "f2m_get_cut_duals", "f2m_solve_subtour"):
        getattr(L, name).restype = C.c_int
    L.f2m_pricing_mma_check.argtypes = [i64, C.c_uint64, C.POINTER(i64), C.POINTER(i64)]
    L.f2m_kernel_launches.argtypes = []
    L.f2m_kernel_launches.restype = C.c_int64
    for name in ("f2m_create", "f2m_set_lambda", "f2m_set_degrees", "f2m_get_colors", "f2m_solve", "f2m_gdp", "f2m_price",
                 "f2m_add_edges", "f2m_extract", "f2m_get_lambda", "f2m_get_bound", "f2m_get_x"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


# ---- marshalling helpers ------------------------------------------------------------

def _ptr(a):
    """(pointer, keepalive) for a numpy array or torch tensor; None passes NULL."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), a
    a = np.ascontiguousarray(a)
    return a.ctypes.data, a


def _as(a, dtype):
    if hasattr(a, "data_ptr"):
        import torch
        tmap = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}
        return a.to(tmap[dtype]).contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def _out(shape, dtype, device):
    if device is None:
        return np.zeros(shape, dtype=dtype)
    import torch
    tmap = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}
    return torch.zeros(shape, dtype=tmap[dtype], device=device)


def _stream_handle(stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Ctx:
    """Owns one f2m_ctx*; destroyed with the object."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.f2m_destroy(self.handle)
            self.handle = None


def _check(ctx, st):
    if st != F2M_OK:
        L = load()
        msg = L.f2m_last_error(ctx.handle if isinstance(ctx, Ctx) else None).decode()
        name = L.f2m_status_string(st).decode()
        raise F2MError(st, f"{name}: {msg}")


# ---- the C ABI, one function each --------------------------------------------------

def f2m_default_params(**overrides) -> f2m_params:
    p = f2m_params()
    load().f2m_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def f2m_create(xy, row_ptr, col, params: f2m_params | None = None, stream=None) -> Ctx:
    L = load()
    xy = _as(xy, np.int32)
    row_ptr = _as(row_ptr, np.int32)
    col = _as(col, np.int32)
    n = int(row_ptr.shape[0]) - 1
    pxy, k1 = _ptr(xy)
    prp, k2 = _ptr(row_ptr)
    pcol, k3 = _ptr(col)
    h = C.c_void_p()
    st = L.f2m_create(pxy, n, prp, pcol, C.byref(params) if params is not None else None,
                      _stream_handle(stream), C.byref(h))
    _check(None, st)
    return Ctx(h.value, n)


def f2m_destroy(ctx: Ctx) -> None:
    if ctx.handle:
        load().f2m_destroy(ctx.handle)
        ctx.handle = None


def f2m_set_lambda(ctx: Ctx, lam, frac_bits: int) -> None:
    p, keep = _ptr(_as(lam, np.int32))
    _check(ctx, load().f2m_set_lambda(ctx.handle, p, frac_bits))


def f2m_set_degrees(ctx: Ctx, b) -> None:
    """Degree requirements b_v (fractional b-matching); a scalar sets every b_v,
    None restores b_v = 2."""
    if b is not None and not hasattr(b, "data_ptr") and np.ndim(b) == 0:
        b = np.full(ctx.n, int(b), np.int32)
    p, keep = _ptr(None if b is None else _as(b, np.int32))
    _check(ctx, load().f2m_set_degrees(ctx.handle, p))


def f2m_get_colors(ctx: Ctx, device=None):
    """Colouring of the class-by-class sweeps: (ncolors, color int32 [n])."""
    color = _out(ctx.n, np.int32, device)
    nc = C.c_int32()
    p, keep = _ptr(color)
    _check(ctx, load().f2m_get_colors(ctx.handle, p, C.byref(nc)))
    return nc.value, color


def f2m_solve(ctx: Ctx, raise_on_error: bool = True) -> f2m_info:
    info = f2m_info()
    st = load().f2m_solve(ctx.handle, C.byref(info))
    if raise_on_error:
        _check(ctx, st)
    return info


def f2m_gdp(ctx: Ctx, max_sweeps: int, trace_cap: int = 0):
    """One GDP phase; returns (status, sweeps, trace_bound2, trace_changed)."""
    sw = C.c_int64()
    tb = np.zeros(max(trace_cap, 1), np.int64)
    tc = np.zeros(max(trace_cap, 1), np.int64)
    st = load().f2m_gdp(ctx.handle, max_sweeps, C.byref(sw), tb.ctypes.data if trace_cap else None,
                        tc.ctypes.data if trace_cap else None, trace_cap)
    if st not in (F2M_OK, F2M_ERR_NOT_CONVERGED, F2M_ERR_OVERFLOW, F2M_ERR_TIMEOUT):
        _check(ctx, st)
    k = min(sw.value, trace_cap)
    return st, sw.value, (tb[:k] if trace_cap else None), (tc[:k] if trace_cap else None)


def f2m_price(ctx: Ctx, cap: int | None = None):
    """Pricing scan; returns (count, pairs int32 [count, 2] in unspecified order)."""
    L = load()
    cnt = C.c_int64()
    _check(ctx, L.f2m_price(ctx.handle, C.byref(cnt), None, 0))
    c = cnt.value
    if cap is not None and c > cap:
        return c, None
    out = np.zeros((max(c, 1), 2), np.int32)
    if c:
        _check(ctx, L.f2m_price(ctx.handle, C.byref(cnt), out.ctypes.data, c))
    return c, out[:c]


def f2m_add_edges(ctx: Ctx, pairs) -> None:
    pairs = _as(pairs, np.int32)
    npairs = int(pairs.shape[0]) if pairs.ndim == 2 else int(pairs.shape[0]) // 2
    p, keep = _ptr(pairs)
    _check(ctx, load().f2m_add_edges(ctx.handle, p, npairs))


def f2m_extract(ctx: Ctx, device=None):
    """Rule (7) extraction at the current lambda; returns (bad_rows, x2)."""
    nnz = C.c_int64(0)
    _check(ctx, load().f2m_get_x(ctx.handle, C.byref(nnz), None, None, None, None))
    x2 = _out((nnz.value,), np.uint8, device)
    p, keep = _ptr(x2)
    bad = C.c_int64()
    _check(ctx, load().f2m_extract(ctx.handle, p, C.byref(bad)))
    return bad.value, x2


def _room(a, count, what):
    """Checks that the caller's output array `a` holds at least `count` entries."""
    size = a.numel() if hasattr(a, "numel") else np.asarray(a).size
    if size < count:
        raise ValueError(f"{what}: the output array holds {size} entries, {count} are needed")
    if not hasattr(a, "data_ptr") and not np.asarray(a).flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what}: the output array must be contiguous")
    return size


def f2m_get_lambda(ctx: Ctx, device=None, out=None):
    """Returns (lambda int32 [n], frac_bits).  out: an int32 array (numpy or a
    torch tensor: host, pinned host or device) of at least n entries to write
    into instead of a new one; the result is its first n entries."""
    if out is not None:
        _room(out, ctx.n, "f2m_get_lambda")
        lam = out[:ctx.n]
    else:
        lam = _out((ctx.n,), np.int32, device)
    p, keep = _ptr(lam)
    fb = C.c_int32()
    _check(ctx, load().f2m_get_lambda(ctx.handle, p, C.byref(fb)))
    return lam, fb.value


def f2m_get_bound(ctx: Ctx):
    """Returns (bound2, frac_bits): 2*LB in units 2^-frac_bits."""
    b = C.c_int64()
    fb = C.c_int32()
    _check(ctx, load().f2m_get_bound(ctx.handle, C.byref(b), C.byref(fb)))
    return b.value, fb.value


def f2m_get_x(ctx: Ctx, device=None, out=None):
    """Returns (row_ptr, col, x2, cost) of the current candidate graph.  out:
    (row_ptr, col, x2, cost) arrays (int32, int32, uint8, int32; numpy or torch
    tensors: host, pinned host or device) to write into instead of new ones,
    row_ptr with n + 1 entries and the others with room for the graph's
    entries; the result is their leading parts."""
    L = load()
    nnz = C.c_int64(0)
    if out is not None:
        rp, col, x2, cost = out
        _room(rp, ctx.n + 1, "f2m_get_x row_ptr")
        nnz.value = min(_room(a, 0, "f2m_get_x") for a in (col, x2, cost))
        rp = rp[:ctx.n + 1]
        ptrs = [_ptr(a) for a in (rp, col, x2, cost)]
        _check(ctx, L.f2m_get_x(ctx.handle, C.byref(nnz), *[p for p, _ in ptrs]))
        m = nnz.value
        return rp, col[:m], x2[:m], cost[:m]
    _check(ctx, L.f2m_get_x(ctx.handle, C.byref(nnz), None, None, None, None))
    rp = _out((ctx.n + 1,), np.int32, device)
    col = _out((nnz.value,), np.int32, device)
    x2 = _out((nnz.value,), np.uint8, device)
    cost = _out((nnz.value,), np.int32, device)
    ptrs = [_ptr(a) for a in (rp, col, x2, cost)]
    _check(ctx, L.f2m_get_x(ctx.handle, C.byref(nnz), *[p for p, _ in ptrs]))
    return rp, col, x2, cost


@dataclass
class Solution:
    info: dict
    row_ptr: np.ndarray
    col: np.ndarray
    x2: np.ndarray
    lam: np.ndarray
    frac_bits: int

    @property
    def opt(self) -> float:
        """The certified optimum as a length: bound2 / (2 * 2^frac_bits)."""
        return self.info["bound2"] / (2.0 * (1 << self.info["frac_bits"]))


def solve(xy, row_ptr, col, lam0=None, params: f2m_params | None = None, stream=None,
          b=None, raise_on_error: bool = True) -> Solution:
    """Create, optionally set degree requirements b (fractional b-matching) and
    warm-start, solve, and read back everything (with raise_on_error False, also
    the state a failed solve stopped in; info["status"] holds its status)."""
    ctx = f2m_create(xy, row_ptr, col, params, stream)
    try:
        if b is not None:
            f2m_set_degrees(ctx, b)
        if lam0 is not None:
            f2m_set_lambda(ctx, lam0, (params.frac_bits if params is not None else 8))
        info = f2m_solve(ctx, raise_on_error)
        rp, c, x2, _ = f2m_get_x(ctx)
        lam, fb = f2m_get_lambda(ctx)
        return Solution(info.as_dict(), rp, c, x2, lam, fb)
    finally:
        f2m_destroy(ctx)


# ---- subtour-elimination cuts --------------------------------------------------------

def f2m_separate(ctx: Ctx, device=None):
    """One cut layer from the x held now: (comp int32 [n], ncuts)."""
    comp = _out((ctx.n,), np.int32, device)
    m = C.c_int32()
    p, _ = _ptr(comp)
    _check(ctx, load().f2m_separate(ctx.handle, p, C.byref(m)))
    return comp, m.value


def f2m_add_cut_layer(ctx: Ctx, comp, ncuts: int) -> None:
    p, keep = _ptr(_as(comp, np.int32))
    _check(ctx, load().f2m_add_cut_layer(ctx.handle, p, int(ncuts)))


def f2m_get_cut_duals(ctx: Ctx):
    """(mu int32 [cuts], layers)."""
    cnt, layers = C.c_int64(0), C.c_int32()
    _check(ctx, load().f2m_get_cut_duals(ctx.handle, None, C.byref(cnt), C.byref(layers)))
    mu = np.zeros(max(cnt.value, 1), np.int32)
    if cnt.value:
        _check(ctx, load().f2m_get_cut_duals(ctx.handle, mu.ctypes.data, C.byref(cnt), None))
    return mu[:cnt.value], layers.value


def f2m_solve_subtour(ctx: Ctx, rounds: int, raise_on_error: bool = True) -> dict:
    info = f2m_subtour_info()
    st = load().f2m_solve_subtour(ctx.handle, int(rounds), C.byref(info))
    if raise_on_error:
        _check(ctx, st)
    return info.as_dict()


def f2m_status_string(status: int) -> str:
    return load().f2m_status_string(status).decode()


def f2m_last_error(ctx: Ctx | None = None) -> str:
    return load().f2m_last_error(ctx.handle if ctx is not None else None).decode()


def f2m_pricing_mma_check(rounds: int, seed: int = 0):
    """Tensor-core arithmetic check of the pricing filter: (values checked, mismatches)."""
    L = load()
    chk, bad = C.c_int64(), C.c_int64()
    _check(None, L.f2m_pricing_mma_check(int(rounds), int(seed), C.byref(chk), C.byref(bad)))
    return chk.value, bad.value


def f2m_kernel_launches() -> int:
    """Kernel launches made by the library so far in this process."""
    return int(load().f2m_kernel_launches())


def f2m_gdp_noalloc(row_ptr, ec, lam, max_sweeps: int, frac_bits: int = 8, damping_shift: int = 2,
                    stream=None):
    """GDP phase without allocation; row_ptr, ec ([nnz, 2] {col, cost}) and lam are
    CUDA tensors, lam is updated in place.  Returns (status, sweeps, bound2, message)."""
    n = int(row_ptr.shape[0]) - 1
    nnz = int(ec.shape[0])
    sw, b2 = C.c_int64(), C.c_int64()
    buf = C.create_string_buffer(512)
    st = load().f2m_gdp_noalloc(row_ptr.data_ptr(), ec.data_ptr(), nnz, n, frac_bits, damping_shift,
                                max_sweeps, lam.data_ptr(), C.byref(sw), C.byref(b2),
                                _stream_handle(stream), buf, len(buf))
    return st, sw.value, b2.value, buf.value.decode()


class Batch:
    """Owns one f2m_batch*; destroyed with the object."""

    def __init__(self, handle, ns):
        self.handle = handle
        self.ns = list(ns)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.f2m_destroy_batch(self.handle)
            self.handle = None


def _bcheck(b, st):
    if st != F2M_OK:
        L = load()
        msg = L.f2m_batch_last_error(b.handle if isinstance(b, Batch) else None)
        name = L.f2m_status_string(st).decode()
        raise F2MError(st, f"{name}: {(msg or b'').decode()}")


def f2m_create_batch(instances, params: f2m_params | None = None, stream=None) -> Batch:
    """instances: list of (xy [n, 2], row_ptr [n + 1], col [nnz]) numpy arrays."""
    L = load()
    ns = np.array([len(rp) - 1 for _, rp, _ in instances], dtype=np.int32)
    xy = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int32).reshape(-1, 2) for x, _, _ in instances]))
    rp = np.ascontiguousarray(np.concatenate([np.asarray(r, np.int32) for _, r, _ in instances]))
    col = np.ascontiguousarray(np.concatenate([np.asarray(c, np.int32) for _, _, c in instances]))
    h = C.c_void_p()
    st = L.f2m_create_batch(len(ns), ns.ctypes.data, xy.ctypes.data, rp.ctypes.data, col.ctypes.data,
                            C.byref(params) if params is not None else None, _stream_handle(stream),
                            C.byref(h))
    if st != F2M_OK:
        raise F2MError(st, f"{L.f2m_status_string(st).decode()}: {L.f2m_last_error(None).decode()}")
    return Batch(h.value, ns)


def f2m_solve_batch(b: Batch, raise_on_error: bool = True):
    """Returns (per-instance f2m_info list, batch total f2m_info)."""
    infos = (f2m_info * len(b.ns))()
    tot = f2m_info()
    st = load().f2m_solve_batch(b.handle, infos, C.byref(tot))
    if raise_on_error:
        _bcheck(b, st)
    return list(infos), tot


def f2m_batch_get_lambda(b: Batch, i: int, out=None):
    """(lambda of instance i, frac_bits); out as in f2m_get_lambda."""
    if out is not None:
        _room(out, b.ns[i], "f2m_batch_get_lambda")
        lam = out[:b.ns[i]]
    else:
        lam = np.zeros(b.ns[i], np.int32)
    p, keep = _ptr(lam)
    fb = C.c_int32()
    _bcheck(b, load().f2m_batch_get_lambda(b.handle, i, p, C.byref(fb)))
    return lam, fb.value


def f2m_batch_get_x(b: Batch, i: int, out=None):
    """(row_ptr, col, x2) of instance i; out: (row_ptr, col, x2) arrays to write
    into, as in f2m_get_x."""
    L = load()
    nnz = C.c_int64(0)
    if out is not None:
        rp, col, x2 = out
        _room(rp, b.ns[i] + 1, "f2m_batch_get_x row_ptr")
        nnz.value = min(_room(a, 0, "f2m_batch_get_x") for a in (col, x2))
        rp = rp[:b.ns[i] + 1]
        ptrs = [_ptr(a) for a in (rp, col, x2)]
        _bcheck(b, L.f2m_batch_get_x(b.handle, i, C.byref(nnz), *[p for p, _ in ptrs]))
        m = nnz.value
        return rp, col[:m], x2[:m]
    _bcheck(b, L.f2m_batch_get_x(b.handle, i, C.byref(nnz), None, None, None))
    rp = np.zeros(b.ns[i] + 1, np.int32)
    col = np.zeros(max(nnz.value, 1), np.int32)
    x2 = np.zeros(max(nnz.value, 1), np.uint8)
    _bcheck(b, L.f2m_batch_get_x(b.handle, i, C.byref(nnz), rp.ctypes.data, col.ctypes.data, x2.ctypes.data))
    return rp, col[:nnz.value], x2[:nnz.value]


def f2m_batch_last_error(b: Batch | None = None) -> str:
    r = load().f2m_batch_last_error(b.handle if b is not None else None)
    return (r or b"").decode()


def f2m_destroy_batch(b: Batch) -> None:
    if b.handle:
        load().f2m_destroy_batch(b.handle)
        b.handle = None


# ---- candidate graph and learned warm start -----------------------------------------

def _gcheck(st):
    if st != F2M_OK:
        L = load()
        raise F2MError(st, f"{L.f2m_status_string(st).decode()}: {L.f2m_last_error(None).decode()}")


def f2m_tsplib_parse(text):
    """TSPLIB EUC_2D problem text -> (xy int32 [n, 2] translated to start at 0,
    (tx, ty) the translation).  Raises F2MError on anything else."""
    data = text.encode() if isinstance(text, str) else bytes(text)
    L = load()
    n = C.c_int32()
    st = L.f2m_tsplib_parse(data, len(data), None, 0, C.byref(n), None)
    if st != F2M_OK:
        raise F2MError(st, L.f2m_tsplib_last_error().decode())
    xy = np.zeros((n.value, 2), np.int32)
    tr = np.zeros(2, np.int64)
    st = L.f2m_tsplib_parse(data, len(data), xy.ctypes.data, n.value, C.byref(n), tr.ctypes.data)
    if st != F2M_OK:
        raise F2MError(st, L.f2m_tsplib_last_error().decode())
    return xy, (int(tr[0]), int(tr[1]))


def f2m_tsplib_last_error() -> str:
    return load().f2m_tsplib_last_error().decode()


def read_tsplib(path):
    """f2m_tsplib_parse of a file."""
    with open(path, "rb") as fh:
        return f2m_tsplib_parse(fh.read())


def f2m_knn(xy, k: int, stream=None, with_d2: bool = True):
    """(nbr int32 [n, k], d2 int64 [n, k] or None): exact k nearest neighbours."""
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    nbr = np.zeros((n, k), np.int32)
    d2 = np.zeros((n, k), np.int64) if with_d2 else None
    _gcheck(load().f2m_knn(xy.ctypes.data, n, k, nbr.ctypes.data,
                           d2.ctypes.data if with_d2 else None, _stream_handle(stream)))
    return nbr, d2


def f2m_knn_csr(xy, k: int, stream=None):
    """(row_ptr, col) of the symmetrised k-NN candidate graph."""
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(2 * n * k, np.int32)
    nnz = C.c_int64()
    _gcheck(load().f2m_knn_csr(xy.ctypes.data, n, k, rp.ctypes.data, col.ctypes.data, C.byref(nnz),
                               _stream_handle(stream)))
    return rp, col[:nnz.value].copy()


def f2m_features(xy, stream=None, device=None):
    """(feat float32 [n, 16], scale float32 [n]) of the warm start; torch tensors
    on `device` when given (xy may then be a CUDA tensor), else numpy."""
    if device is not None:
        import torch
        xy_t = torch.as_tensor(np.asarray(xy, np.int32) if not hasattr(xy, "data_ptr") else xy,
                               device=device).to(torch.int32).contiguous()
        n = int(xy_t.shape[0])
        feat = torch.zeros((n, 16), dtype=torch.float32, device=device)
        scale = torch.zeros(n, dtype=torch.float32, device=device)
        _gcheck(load().f2m_features(xy_t.data_ptr(), n, feat.data_ptr(), scale.data_ptr(),
                                    _stream_handle(stream)))
        return feat, scale
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    feat = np.zeros((n, 16), np.float32)
    scale = np.zeros(n, np.float32)
    _gcheck(load().f2m_features(xy.ctypes.data, n, feat.ctypes.data, scale.ctypes.data,
                                _stream_handle(stream)))
    return feat, scale


class Mlp:
    """Owns one f2m_mlp*; destroyed with the object."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.f2m_mlp_destroy(self.handle)
            self.handle = None


def _mcheck(m, st):
    if st != F2M_OK:
        L = load()
        msg = L.f2m_mlp_last_error(m.handle) if isinstance(m, Mlp) else L.f2m_last_error(None)
        raise F2MError(st, f"{L.f2m_status_string(st).decode()}: {(msg or b'').decode()}")


def f2m_mlp_create(params, stream=None) -> Mlp:
    L = load()
    p, keep = _ptr(params if hasattr(params, "data_ptr") else np.asarray(params, np.float32))
    h = C.c_void_p()
    st = L.f2m_mlp_create(p, _stream_handle(stream), C.byref(h))
    _mcheck(None, st)
    return Mlp(h.value)


def f2m_mlp_destroy(m: Mlp) -> None:
    if m.handle:
        load().f2m_mlp_destroy(m.handle)
        m.handle = None


def f2m_mlp_get_params(m: Mlp) -> np.ndarray:
    out = np.zeros(F2M_MLP_NPARAMS, np.float32)
    _mcheck(m, load().f2m_mlp_get_params(m.handle, out.ctypes.data))
    return out


def f2m_mlp_last_error(m: Mlp) -> str:
    return (load().f2m_mlp_last_error(m.handle) or b"").decode()


def f2m_mlp_forward(m: Mlp, feat):
    """y [count]: numpy for numpy input, a CUDA tensor for a CUDA tensor input."""
    if hasattr(feat, "data_ptr"):
        import torch
        feat = feat.to(torch.float32).contiguous()
        y = torch.zeros(feat.shape[0], dtype=torch.float32, device=feat.device)
        _mcheck(m, load().f2m_mlp_forward(m.handle, feat.data_ptr(), feat.shape[0], y.data_ptr()))
        return y
    feat = np.ascontiguousarray(feat, np.float32)
    y = np.zeros(feat.shape[0], np.float32)
    _mcheck(m, load().f2m_mlp_forward(m.handle, feat.ctypes.data, feat.shape[0], y.ctypes.data))
    return y


def f2m_mlp_grad(m: Mlp, feat, target):
    """(loss, grad float32 [F2M_MLP_NPARAMS]) of the mean squared error."""
    fp, kf = _ptr(feat if hasattr(feat, "data_ptr") else np.asarray(feat, np.float32))
    tp, kt = _ptr(target if hasattr(target, "data_ptr") else np.asarray(target, np.float32))
    grad = np.zeros(F2M_MLP_NPARAMS, np.float32)
    loss = np.zeros(1, np.float32)
    _mcheck(m, load().f2m_mlp_grad(m.handle, fp, tp, int(feat.shape[0]), grad.ctypes.data, loss.ctypes.data))
    return float(loss[0]), grad


def f2m_mlp_train(m: Mlp, feat, target, epochs: int = 1, batch: int = 38912, lr: float = 1e-3,
                  lr_final_frac: float = 1.0, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                  seed: int = 0):
    """Trains in place; returns the mean loss of each epoch (numpy float32)."""
    fp, kf = _ptr(feat if hasattr(feat, "data_ptr") else np.asarray(feat, np.float32))
    tq, kt = _ptr(target if hasattr(target, "data_ptr") else np.asarray(target, np.float32))
    tpar = f2m_train_params(epochs, batch, lr, lr_final_frac, beta1, beta2, eps, seed)
    out = np.zeros(max(epochs, 1), np.float32)
    _mcheck(m, load().f2m_mlp_train(m.handle, fp, tq, int(feat.shape[0]), C.byref(tpar), out.ctypes.data))
    return out[:epochs]


def f2m_warm_start(ctx: Ctx, m: Mlp) -> float:
    """Sets the context's lambda from the network; returns the device ms it took."""
    ms = C.c_double()
    _check(ctx, load().f2m_warm_start(ctx.handle, m.handle, C.byref(ms)))
    return ms.value
