"""Thin ctypes binding of the C ABI in ``include/nncp.h`` (argument marshalling only).

Every compute step runs in the CUDA library ``_lib/libnncp.so``; this module
only converts Python/torch arguments to pointers and sizes.  Loading fails
loudly if the library has not been built: there is no fallback.

Functions keep the C names (``nncp_create``, ``nncp_mttkrp`` ...).  ``Context``
is a small convenience wrapper that allocates the workspace with torch.
"""

from __future__ import annotations

import ctypes
import math
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libnncp.so")

NNCP_OK = 0
NNCP_ERR_INVALID_ARG = 1
NNCP_ERR_OUT_OF_MEMORY = 2
NNCP_ERR_CUDA = 3
NNCP_ERR_NUMERIC = 4
NNCP_ERR_TIMEOUT = 5
NNCP_ERR_NOT_READY = 6
NNCP_ERR_UNSUPPORTED = 7

NNCP_FP32_SIMT = 0
NNCP_TF32 = 1
NNCP_SPLIT_BF16X3 = 2
NNCP_BF16_STORED = 3

PRECISIONS = {"fp32_simt": NNCP_FP32_SIMT, "tf32": NNCP_TF32,
              "split_bf16x3": NNCP_SPLIT_BF16X3, "bf16_stored": NNCP_BF16_STORED}

_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_dblp = ctypes.POINTER(ctypes.c_double)
_c_intp = ctypes.POINTER(ctypes.c_int)
_c_vpp = ctypes.POINTER(ctypes.c_void_p)

# (name, restype, argtypes)
_SIGNATURES = [
    ("nncp_version", ctypes.c_char_p, []),
    ("nncp_default_split", ctypes.c_int, [ctypes.c_int, _c_i64p]),
    ("nncp_create", ctypes.c_int, [ctypes.c_int, _c_i64p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("nncp_set_options", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("nncp_set_dimtree", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("nncp_set_leaf_fusion", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("nncp_set_nls", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("nncp_set_nls_iters", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("nncp_solve_host_release", None, []),
    ("nncp_workspace_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("nncp_set_workspace", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("nncp_set_tensor", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("nncp_set_factors", ctypes.c_int, [ctypes.c_void_p, _c_vpp]),
    ("nncp_mttkrp", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("nncp_partial_mttkrp", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("nncp_mttkrp_cached", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("nncp_factor_changed", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("nncp_iteration_kernels", ctypes.c_int, [ctypes.c_void_p, _c_intp]),
    ("nncp_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_vpp, _c_dblp, ctypes.c_int,
                                  ctypes.c_double, _c_intp, _c_dblp]),
    ("nncp_solve_bound", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _c_dblp,
                                        _c_intp, _c_dblp]),
    ("nncp_fit_history", ctypes.c_int, [ctypes.c_void_p, _c_dblp, ctypes.c_int, _c_intp]),
    ("nncp_fit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_dblp]),
    ("nncp_solve_begin", ctypes.c_int, [ctypes.c_void_p]),
    ("nncp_iterate", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("nncp_tensor_to_bf16", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    ("nncp_solve_host", ctypes.c_int, [ctypes.c_int, _c_i64p, ctypes.c_int, ctypes.c_void_p, _c_vpp,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       _c_dblp, _c_intp, _c_dblp]),
    ("nncp_mttkrp_noalloc", ctypes.c_int, [ctypes.c_int, _c_i64p, ctypes.c_int, ctypes.c_void_p,
                                           _c_vpp, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("nncp_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _c_i64p, _c_intp, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    ("nncp_batch_workspace_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("nncp_batch_set_workspace", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("nncp_batch_set_data", ctypes.c_int, [ctypes.c_void_p, _c_vpp, _c_vpp]),
    ("nncp_batch_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _c_intp, _c_dblp,
                                      _c_dblp, ctypes.c_void_p]),
    ("nncp_batch_solve", ctypes.c_int, [ctypes.c_int, _c_intp, ctypes.POINTER(_c_i64p), _c_intp,
                                        _c_vpp, ctypes.POINTER(_c_vpp), ctypes.POINTER(_c_dblp),
                                        ctypes.c_int, ctypes.c_double, _c_intp, _c_dblp,
                                        ctypes.c_void_p]),
    ("nncp_batch_set_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("nncp_batch_set_wait_limit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    ("nncp_batch_get_schedule", ctypes.c_int, [ctypes.c_void_p, _c_intp, _c_intp]),
    ("nncp_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("nncp_batch_destroy", None, [ctypes.c_void_p]),
    ("nncp_server_create", ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("nncp_server_create_ex", ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("nncp_server_footprint", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_i64p, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("nncp_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    ("nncp_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    ("nncp_server_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]),
    ("nncp_server_release", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("nncp_server_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("nncp_server_clock", ctypes.c_double, [ctypes.c_void_p]),
    ("nncp_server_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("nncp_server_destroy", None, [ctypes.c_void_p]),
    ("nncp_peak_probe", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       _c_dblp]),
    ("nncp_par_create", ctypes.c_int, [ctypes.c_int, _c_i64p, _c_intp, _c_intp, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("nncp_par_layout", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_i64p, _c_i64p, _c_i64p,
                                       _c_i64p, _c_intp, _c_intp]),
    ("nncp_par_workspace_size", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("nncp_par_set_workspace", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                              ctypes.c_void_p]),
    ("nncp_par_set_data", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_vpp]),
    ("nncp_par_alpha_local", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_dblp]),
    ("nncp_par_begin", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]),
    ("nncp_par_mttkrp", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("nncp_par_update", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p, _c_dblp]),
    ("nncp_par_normalize", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_dblp, ctypes.c_void_p,
                                          ctypes.c_int, _c_dblp, _c_intp]),
    ("nncp_par_result", ctypes.c_int, [ctypes.c_void_p, _c_dblp, _c_dblp, ctypes.c_int, _c_intp]),
    ("nncp_par_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("nncp_par_destroy", None, [ctypes.c_void_p]),
    ("nncp_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("nncp_global_error", ctypes.c_char_p, []),
    ("nncp_destroy", None, [ctypes.c_void_p]),
]

_lib = None


def exported_symbols():
    return [name for name, _, _ in _SIGNATURES]


def load(path=LIB_PATH):
    """Load the library (once).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"NNCP CUDA library not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class NNCPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"nncp status {status}: {msg}")
        self.status = status


def _check(status, ctx=None):
    if status != NNCP_OK:
        lib = load()
        msg = lib.nncp_last_error(ctx) if ctx else lib.nncp_global_error()
        raise NNCPError(status, (msg or b"").decode())


def _dims(dims):
    return (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else int(t.data_ptr()))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


# ---- functions with the C names ------------------------------------------------

def nncp_version():
    return load().nncp_version().decode()


def nncp_default_split(dims):
    return load().nncp_default_split(len(dims), _dims(dims))


def nncp_create(dims, R):
    ctx = ctypes.c_void_p()
    _check(load().nncp_create(len(dims), _dims(dims), int(R), ctypes.byref(ctx)))
    return ctx


def nncp_set_options(ctx, precision=NNCP_FP32_SIMT, root_split=0, stream=None):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    _check(load().nncp_set_options(ctx, int(precision), int(root_split), _stream(stream)), ctx)


def nncp_set_dimtree(ctx, enabled):
    _check(load().nncp_set_dimtree(ctx, 1 if enabled else 0), ctx)


def nncp_set_leaf_fusion(ctx, enabled):
    _check(load().nncp_set_leaf_fusion(ctx, 1 if enabled else 0), ctx)


NNCP_NLS_HALS, NNCP_NLS_BPP, NNCP_NLS_ADMM, NNCP_NLS_APG = 0, 1, 2, 3
NLS = {"hals": NNCP_NLS_HALS, "bpp": NNCP_NLS_BPP, "admm": NNCP_NLS_ADMM, "apg": NNCP_NLS_APG}


def nncp_set_nls(ctx, nls):
    if isinstance(nls, str):
        if nls not in NLS:
            raise ValueError(f"unknown NLS update {nls!r}; one of {sorted(NLS)}")
        nls = NLS[nls]
    _check(load().nncp_set_nls(ctx, int(nls)), ctx)


def nncp_set_nls_iters(ctx, iters):
    _check(load().nncp_set_nls_iters(ctx, int(iters)), ctx)


def nncp_workspace_size(ctx):
    n = ctypes.c_size_t()
    _check(load().nncp_workspace_size(ctx, ctypes.byref(n)), ctx)
    return n.value


def nncp_set_workspace(ctx, ws):
    _check(load().nncp_set_workspace(ctx, _ptr(ws), ws.numel() * ws.element_size()), ctx)


def nncp_set_tensor(ctx, X):
    _check(load().nncp_set_tensor(ctx, _ptr(X)), ctx)


def nncp_set_factors(ctx, H):
    arr = (ctypes.c_void_p * len(H))(*[int(h.data_ptr()) for h in H])
    _check(load().nncp_set_factors(ctx, arr), ctx)


def nncp_mttkrp(ctx, mode, use_dimtree, M):
    _check(load().nncp_mttkrp(ctx, int(mode), int(use_dimtree), _ptr(M)), ctx)


def nncp_partial_mttkrp(ctx, side, T):
    _check(load().nncp_partial_mttkrp(ctx, int(side), _ptr(T)), ctx)


def nncp_mttkrp_cached(ctx, mode, M):
    _check(load().nncp_mttkrp_cached(ctx, int(mode), _ptr(M)), ctx)


def nncp_factor_changed(ctx, mode):
    _check(load().nncp_factor_changed(ctx, int(mode)), ctx)


def nncp_iteration_kernels(ctx):
    n = ctypes.c_int()
    _check(load().nncp_iteration_kernels(ctx, ctypes.byref(n)), ctx)
    return n.value


def nncp_solve(ctx, R, X, H, max_iters, tol):
    """Solve on the device tensor X and factors H (None keeps the bound ones);
    returns (lambda, iterations, fit)."""
    lam = (ctypes.c_double * R)()
    iters = ctypes.c_int()
    fit = ctypes.c_double()
    harr = None if H is None else (ctypes.c_void_p * len(H))(*[int(h.data_ptr()) for h in H])
    _check(load().nncp_solve(ctx, _ptr(X), harr, lam, int(max_iters), float(tol),
                             ctypes.byref(iters), ctypes.byref(fit)), ctx)
    return list(lam), iters.value, fit.value


def nncp_solve_bound(ctx, R, max_iters, tol):
    lam = (ctypes.c_double * R)()
    iters = ctypes.c_int()
    fit = ctypes.c_double()
    _check(load().nncp_solve_bound(ctx, int(max_iters), float(tol), lam, ctypes.byref(iters),
                                   ctypes.byref(fit)), ctx)
    return list(lam), iters.value, fit.value


def nncp_fit_history(ctx, max_count):
    buf = (ctypes.c_double * max_count)()
    n = ctypes.c_int()
    _check(load().nncp_fit_history(ctx, buf, int(max_count), ctypes.byref(n)), ctx)
    return list(buf[: n.value])


def nncp_fit(ctx, exact=False):
    f = ctypes.c_double()
    _check(load().nncp_fit(ctx, int(bool(exact)), ctypes.byref(f)), ctx)
    return f.value


def nncp_solve_begin(ctx):
    _check(load().nncp_solve_begin(ctx), ctx)


def nncp_iterate(ctx, iters):
    _check(load().nncp_iterate(ctx, int(iters)), ctx)


def nncp_tensor_to_bf16(X, Xb, stream=None):
    _check(load().nncp_tensor_to_bf16(_ptr(X), _ptr(Xb), X.numel(), _stream(stream)))


def nncp_solve_host_release():
    """Frees the plan (context, graphs, device buffers) nncp_solve_host keeps."""
    load().nncp_solve_host_release()


def nncp_solve_host(dims, R, X_host, H_host, precision=NNCP_FP32_SIMT, root_split=0,
                    max_iters=50, tol=0.0):
    """X_host: contiguous float32 numpy/torch CPU array; H_host: list of writable
    contiguous float32 (I_n, R) arrays, overwritten with the result."""
    def addr(a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return a.ctypes.data
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    arr = (ctypes.c_void_p * len(H_host))(*[addr(h) for h in H_host])
    lam = (ctypes.c_double * R)()
    iters = ctypes.c_int()
    fit = ctypes.c_double()
    _check(load().nncp_solve_host(len(dims), _dims(dims), int(R), ctypes.c_void_p(addr(X_host)),
                                  arr, int(precision), int(root_split), int(max_iters),
                                  float(tol), lam, ctypes.byref(iters), ctypes.byref(fit)))
    return list(lam), iters.value, fit.value


def nncp_mttkrp_noalloc(dims, R, X, H, mode, M, stream=None):
    """Direct MTTKRP of `mode` (1-based) that allocates nothing on the device.

    X (prod(dims) float32), H[n] ((dims[n], R) float32) and M ((dims[mode-1], R)
    float32) are caller-owned, contiguous CUDA tensors on one device; the C
    side reads exactly those extents, so they are checked here first.  The
    call is asynchronous on `stream` (default: torch's current stream)."""
    import torch
    dims = [int(d) for d in dims]
    R = int(R)
    if not 1 <= int(mode) <= len(dims):
        raise ValueError(f"mode {mode} not in [1, {len(dims)}]")
    if len(H) != len(dims):
        raise ValueError(f"{len(H)} factors for an order-{len(dims)} tensor")

    def need(t, name, shape):
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous float32")
        if t.device != X.device:
            raise ValueError(f"{name} is on {t.device}, X on {X.device}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")

    need(X, "X", None)
    if X.numel() != math.prod(dims):
        raise ValueError(f"X has {X.numel()} elements, dims give {math.prod(dims)}")
    for n, h in enumerate(H):
        need(h, f"H[{n}]", (dims[n], R))
    need(M, "M", (dims[int(mode) - 1], R))
    if stream is None:
        with torch.cuda.device(X.device):
            stream = torch.cuda.current_stream()
    arr = (ctypes.c_void_p * len(H))(*[int(h.data_ptr()) for h in H])
    with torch.cuda.device(X.device):
        _check(load().nncp_mttkrp_noalloc(len(dims), _dims(dims), R, _ptr(X), arr, int(mode),
                                          _ptr(M), _stream(stream)))


def nncp_batch_solve(shapes, ranks, X, H, max_iters, tol, stream=None):
    """One-call batched solve of independent problems of any orders.

    shapes[t]: mode lengths of tensor t; ranks[t]: its rank; X[t]: its CUDA
    tensor; H[t]: its list of CUDA factors, overwritten with the result.
    Returns (iters, fits, lambdas) lists."""
    count = len(shapes)
    Ns = (ctypes.c_int * count)(*[len(sh) for sh in shapes])
    dim_arrs = [_dims(sh) for sh in shapes]
    dims = (_c_i64p * count)(*[ctypes.cast(d, _c_i64p) for d in dim_arrs])
    Rs = (ctypes.c_int * count)(*[int(r) for r in ranks])
    xs = (ctypes.c_void_p * count)(*[int(x.data_ptr()) for x in X])
    h_arrs = [(ctypes.c_void_p * len(h))(*[int(f.data_ptr()) for f in h]) for h in H]
    hs = (_c_vpp * count)(*[ctypes.cast(a, _c_vpp) for a in h_arrs])
    lam_arrs = [(ctypes.c_double * int(r))() for r in ranks]
    lams = (_c_dblp * count)(*[ctypes.cast(a, _c_dblp) for a in lam_arrs])
    iters = (ctypes.c_int * count)()
    fits = (ctypes.c_double * count)()
    _check(load().nncp_batch_solve(count, Ns, dims, Rs, xs, hs, lams, int(max_iters), float(tol),
                                   iters, fits, _stream(stream)))
    return list(iters), list(fits), [list(a) for a in lam_arrs]


PROBES = {"ffma": 0, "tf32": 1, "bf16": 2, "ffma2": 3}


def nncp_peak_probe(kind, reps, sink, stream=None):
    """Launch one throughput probe (kind "ffma", "tf32", "bf16" or "ffma2"; see the
    header); returns the floating-point operations it performs.  sink: a
    CUDA tensor of at least 16 bytes."""
    flops = ctypes.c_double()
    _check(load().nncp_peak_probe(PROBES.get(kind, kind), int(reps), _ptr(sink), _stream(stream),
                                  ctypes.byref(flops)))
    return flops.value


def _bcheck(status, b):
    if status != NNCP_OK:
        lib = load()
        msg = lib.nncp_batch_last_error(b) if b else lib.nncp_global_error()
        raise NNCPError(status, (msg or b"").decode())


class Batch:
    """Batched solver over torch CUDA tensors (argument marshalling only).

    shapes: list of per-tensor mode-length tuples (all of one order N);
    ranks: list of per-tensor ranks.  The workspace is allocated with torch."""

    def __init__(self, shapes, ranks, max_iters):
        import torch
        self.N = len(shapes[0])
        self.count = len(shapes)
        self.ranks = [int(r) for r in ranks]
        flat = [int(d) for sh in shapes for d in sh]
        dims = (ctypes.c_int64 * len(flat))(*flat)
        R = (ctypes.c_int * self.count)(*self.ranks)
        self.b = ctypes.c_void_p()
        _bcheck(load().nncp_batch_create(self.count, self.N, dims, R, int(max_iters),
                                         ctypes.byref(self.b)), None)
        n = ctypes.c_size_t()
        _bcheck(load().nncp_batch_workspace_size(self.b, ctypes.byref(n)), self.b)
        self.ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device="cuda")
        _bcheck(load().nncp_batch_set_workspace(self.b, _ptr(self.ws), n.value), self.b)

    def set_data(self, X, H):
        """X: list of count tensors; H: list of count lists of N factor tensors."""
        self._keep = (list(X), [list(h) for h in H])
        xs = (ctypes.c_void_p * self.count)(*[int(x.data_ptr()) for x in X])
        hs = (ctypes.c_void_p * (self.count * self.N))(*[int(f.data_ptr()) for h in H for f in h])
        _bcheck(load().nncp_batch_set_data(self.b, xs, hs), self.b)

    def solve(self, max_iters, tol, stream=None):
        iters = (ctypes.c_int * self.count)()
        fits = (ctypes.c_double * self.count)()
        lam = (ctypes.c_double * max(1, sum(self.ranks)))()
        _bcheck(load().nncp_batch_run(self.b, int(max_iters), float(tol), iters, fits, lam,
                                      _stream(stream)), self.b)
        lams, o = [], 0
        for r in self.ranks:
            lams.append(list(lam[o:o + r]))
            o += r
        return list(iters), list(fits), lams

    def set_schedule(self, pm_right=-1, pm_left=-1):
        """Root-phase schedules: 0 one CTA per item, 1 persistent, 2 persistent
        and streamed through shared-memory rings by warp roles, -1 tuned."""
        _bcheck(load().nncp_batch_set_schedule(self.b, int(pm_right), int(pm_left)), self.b)

    def set_wait_limit(self, cycles=0):
        """Bounded-wait limit of the streamed kernel in SM cycles (0: the default,
        about two seconds); a test hook for the timeout path."""
        _bcheck(load().nncp_batch_set_wait_limit(self.b, int(cycles)), self.b)

    def schedule(self):
        r, l = ctypes.c_int(), ctypes.c_int()
        _bcheck(load().nncp_batch_get_schedule(self.b, ctypes.byref(r), ctypes.byref(l)), self.b)
        return r.value, l.value

    def close(self):
        if self.b:
            load().nncp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("dims", _c_i64p), ("R", ctypes.c_int),
                ("X_host", ctypes.c_void_p), ("H_init_host", _c_vpp),
                ("max_iters", ctypes.c_int), ("tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("borrow_x", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("fit", ctypes.c_double),
                ("lam", _c_dblp), ("H", ctypes.POINTER(ctypes.POINTER(ctypes.c_float))),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("sweeps", ctypes.c_uint64), ("active", ctypes.c_int), ("queued", ctypes.c_int),
                ("peak_active", ctypes.c_int), ("budget", ctypes.c_size_t),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes_in_use", ctypes.c_size_t)]


class Server:
    """Serving loop over host numpy arrays (argument marshalling only).

    submit() copies the request into the library and returns a ticket;
    poll()/wait() return None / raise TimeoutError until the request is done,
    then a dict with the status, iterations, fit, lambda, factors (numpy
    copies) and the submit/admit/done times on the server clock."""

    SOLO_ELEMS = 1 << 22   # NNCP_SERVER_SOLO_ELEMS
    MAX_SOLO = 2           # NNCP_SERVER_MAX_SOLO

    def __init__(self, hbm_budget_bytes, max_slots, solo_elems=None, max_solo=None):
        self.s = ctypes.c_void_p()
        if solo_elems is None and max_solo is None:
            _scheck(load().nncp_server_create(int(hbm_budget_bytes), int(max_slots),
                                              ctypes.byref(self.s)), None)
        else:
            _scheck(load().nncp_server_create_ex(
                int(hbm_budget_bytes), int(max_slots),
                int(self.SOLO_ELEMS if solo_elems is None else solo_elems),
                int(self.MAX_SOLO if max_solo is None else max_solo), ctypes.byref(self.s)), None)
        self._shapes = {}
        self._borrowed = {}  # ticket -> X the server may still read (borrow=True)

    def footprint(self, dims, R, max_iters, precision=NNCP_FP32_SIMT):
        """Device bytes the request would take from the pool (its lane's layout)."""
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        n = ctypes.c_size_t()
        _scheck(load().nncp_server_footprint(self.s, len(dims), _dims(dims), int(R), int(max_iters),
                                             int(precision), ctypes.byref(n)), self.s)
        return n.value

    def submit(self, dims, R, X, H, max_iters, tol, precision=NNCP_FP32_SIMT, borrow=False):
        """X: host float32 tensor (numpy array or CPU torch tensor).  borrow=True
        passes borrow_x: the server uploads from X itself at admission (page-locked
        memory makes that an asynchronous copy); X is kept referenced here until
        the request's result has been returned or released."""
        import numpy as np
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        if hasattr(X, "data_ptr"):
            if X.device.type != "cpu" or not X.is_contiguous() or X.element_size() != 4:
                raise ValueError("X must be a contiguous float32 CPU tensor")
            xptr = X.data_ptr()
        else:
            X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1)
            xptr = X.ctypes.data
        H = [np.ascontiguousarray(h, dtype=np.float32) for h in H]
        d = _dims(dims)
        hp = (ctypes.c_void_p * len(H))(*[h.ctypes.data for h in H])
        req = _Request(len(dims), ctypes.cast(d, _c_i64p), int(R), xptr,
                       ctypes.cast(hp, _c_vpp), int(max_iters), float(tol), int(precision),
                       1 if borrow else 0)
        t = ctypes.c_uint64()
        _scheck(load().nncp_server_submit(self.s, ctypes.byref(req), ctypes.byref(t)), self.s)
        self._shapes[t.value] = (tuple(int(x) for x in dims), int(R))
        if borrow:
            self._borrowed[t.value] = X
        return t.value

    def _result(self, ticket, res):
        import numpy as np
        self._borrowed.pop(ticket, None)  # done: the server no longer reads X
        dims, R = self._shapes[ticket]
        H = [np.ctypeslib.as_array(res.H[n], shape=(dims[n], R)).copy() for n in range(len(dims))]
        lam = np.ctypeslib.as_array(res.lam, shape=(R,)).copy() if res.lam else None
        return {"status": res.status, "iters": res.iters, "fit": res.fit, "lambda": lam, "H": H,
                "t_submit": res.t_submit, "t_admit": res.t_admit, "t_done": res.t_done}

    def poll(self, ticket):
        res = _Result()
        st = load().nncp_server_poll(self.s, ticket, ctypes.byref(res))
        if st == NNCP_ERR_NOT_READY:
            return None
        _scheck(st, self.s)
        return self._result(ticket, res)

    def wait(self, ticket, timeout_ms):
        res = _Result()
        st = load().nncp_server_wait(self.s, ticket, int(timeout_ms), ctypes.byref(res))
        if st == NNCP_ERR_TIMEOUT:
            raise TimeoutError(f"request {ticket} not done after {timeout_ms} ms")
        _scheck(st, self.s)
        return self._result(ticket, res)

    def release(self, ticket):
        _scheck(load().nncp_server_release(self.s, ticket), self.s)
        self._shapes.pop(ticket, None)
        self._borrowed.pop(ticket, None)

    def stats(self):
        st = _Stats()
        _scheck(load().nncp_server_get_stats(self.s, ctypes.byref(st)), self.s)
        return {k: getattr(st, k) for k, _ in _Stats._fields_}

    def clock(self):
        return load().nncp_server_clock(self.s)

    def close(self):
        if self.s:
            load().nncp_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _scheck(status, s):
    if status != NNCP_OK:
        lib = load()
        msg = lib.nncp_server_last_error(s) if s else lib.nncp_global_error()
        raise NNCPError(status, (msg or b"").decode())


def _pcheck(status, p):
    if status != NNCP_OK:
        lib = load()
        msg = lib.nncp_par_last_error(p) if p else lib.nncp_global_error()
        raise NNCPError(status, (msg or b"").decode())


class ParRank:
    """One processor of a Par-NNCP grid (nncp_par_*; argument marshalling only).

    The local computation between the collectives of Alg. 2: see the
    nncp_par_* declarations for the protocol.  The workspace is allocated with
    torch on the current CUDA device."""

    def __init__(self, dims, grid, coords, R, precision=NNCP_FP32_SIMT, stream=None):
        import torch
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.N, self.R = len(dims), int(R)
        self.p = ctypes.c_void_p()
        g = (ctypes.c_int * self.N)(*[int(v) for v in grid])
        c = (ctypes.c_int * self.N)(*[int(v) for v in coords])
        _pcheck(load().nncp_par_create(self.N, _dims(dims), g, c, self.R, int(precision),
                                       ctypes.byref(self.p)), None)
        n = ctypes.c_size_t()
        _pcheck(load().nncp_par_workspace_size(self.p, ctypes.byref(n)), self.p)
        self.ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device="cuda")
        _pcheck(load().nncp_par_set_workspace(self.p, _ptr(self.ws), n.value, _stream(stream)),
                self.p)

    def layout(self, mode):
        """(block_lo, block_rows, owned_lo, owned_rows, slice_index, slice_size)."""
        v = [ctypes.c_int64() for _ in range(4)] + [ctypes.c_int() for _ in range(2)]
        _pcheck(load().nncp_par_layout(self.p, int(mode), *[ctypes.byref(x) for x in v]), self.p)
        return tuple(x.value for x in v)

    def set_data(self, X_local, H_block):
        self._keep = (X_local, list(H_block))
        arr = (ctypes.c_void_p * len(H_block))(*[int(h.data_ptr()) for h in H_block])
        _pcheck(load().nncp_par_set_data(self.p, _ptr(X_local), arr), self.p)

    def alpha_local(self, X_local):
        a = ctypes.c_double()
        _pcheck(load().nncp_par_alpha_local(self.p, _ptr(X_local), ctypes.byref(a)), self.p)
        return a.value

    def begin(self, alpha, tol):
        _pcheck(load().nncp_par_begin(self.p, float(alpha), float(tol)), self.p)

    def mttkrp(self, mode, M_block):
        _pcheck(load().nncp_par_mttkrp(self.p, int(mode), _ptr(M_block)), self.p)

    def update(self, mode, M_owned, H_owned):
        part = (ctypes.c_double * (self.R * self.R + 1))()
        _pcheck(load().nncp_par_update(self.p, int(mode), _ptr(M_owned), _ptr(H_owned), part),
                self.p)
        return list(part)

    def normalize(self, mode, sums, H_owned, init):
        arr = (ctypes.c_double * len(sums))(*[float(v) for v in sums])
        fit = ctypes.c_double()
        stop = ctypes.c_int()
        _pcheck(load().nncp_par_normalize(self.p, int(mode), arr, _ptr(H_owned), int(bool(init)),
                                          ctypes.byref(fit), ctypes.byref(stop)), self.p)
        return fit.value, bool(stop.value)

    def result(self, max_fits=1 << 16):
        lam = (ctypes.c_double * self.R)()
        fits = (ctypes.c_double * max_fits)()
        n = ctypes.c_int()
        _pcheck(load().nncp_par_result(self.p, lam, fits, int(max_fits), ctypes.byref(n)), self.p)
        return list(lam), list(fits[: n.value])

    def close(self):
        if self.p:
            load().nncp_par_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nncp_last_error(ctx):
    return load().nncp_last_error(ctx).decode()


def nncp_destroy(ctx):
    load().nncp_destroy(ctx)


# ---- convenience wrapper ---------------------------------------------------------

class Context:
    """A context plus a torch-allocated workspace on the current CUDA device."""

    def __init__(self, dims, R, precision=NNCP_FP32_SIMT, root_split=0, stream=None):
        import torch
        self.dims = tuple(int(d) for d in dims)
        self.R = int(R)
        self.ctx = nncp_create(self.dims, self.R)
        self._keep = []
        try:
            nncp_set_options(self.ctx, precision, root_split, stream)
            nbytes = nncp_workspace_size(self.ctx)
            self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
            nncp_set_workspace(self.ctx, self.ws)
        except Exception:
            nncp_destroy(self.ctx)
            self.ctx = None
            raise

    def set_tensor(self, X):
        self._keep = [X] + self._keep[1:] if self._keep else [X]
        nncp_set_tensor(self.ctx, X)

    def set_factors(self, H):
        self._factors = list(H)
        nncp_set_factors(self.ctx, self._factors)

    def mttkrp(self, mode, use_dimtree, out):
        nncp_mttkrp(self.ctx, mode, use_dimtree, out)
        return out

    def partial_mttkrp(self, side, out):
        nncp_partial_mttkrp(self.ctx, side, out)
        return out

    def mttkrp_cached(self, mode, out):
        nncp_mttkrp_cached(self.ctx, mode, out)
        return out

    def factor_changed(self, mode):
        nncp_factor_changed(self.ctx, mode)

    def iteration_kernels(self):
        return nncp_iteration_kernels(self.ctx)

    def set_dimtree(self, enabled):
        nncp_set_dimtree(self.ctx, enabled)

    def set_leaf_fusion(self, enabled):
        nncp_set_leaf_fusion(self.ctx, enabled)

    def set_nls(self, nls):
        nncp_set_nls(self.ctx, nls)

    def set_nls_iters(self, iters):
        nncp_set_nls_iters(self.ctx, iters)

    def solve(self, max_iters, tol=0.0):
        return nncp_solve_bound(self.ctx, self.R, max_iters, tol)

    def solve_on(self, X, H, max_iters, tol=0.0):
        """nncp_solve with the tensor and factors passed in the call."""
        self._keep = [X] + self._keep[1:] if self._keep else [X]
        self._factors = list(H)
        return nncp_solve(self.ctx, self.R, X, self._factors, max_iters, tol)

    def fit_history(self, max_count=1 << 16):
        return nncp_fit_history(self.ctx, max_count)

    def fit(self, exact=False):
        return nncp_fit(self.ctx, exact)

    def solve_begin(self):
        nncp_solve_begin(self.ctx)

    def iterate(self, iters):
        nncp_iterate(self.ctx, iters)

    def close(self):
        if self.ctx is not None:
            nncp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
