"""Thin ctypes binding of the C ABI in include/espnmf.h.

Argument marshalling only: every step of the factorisation runs in the CUDA
library.  Functions keep the ABI's names.  Arrays may be numpy arrays (host
memory) or torch tensors (host or CUDA memory); torch supplies device memory
and streams.  A non-OK status raises EspnmfError.  There is no fallback: if
the library has not been built, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "BAD_MATRIX", 3: "SINGULAR",
                4: "NONFINITE", 5: "OOM", 6: "CUDA", 7: "TIMEOUT", 8: "UNSUPPORTED"}
ERR_INVALID_ARG, ERR_BAD_MATRIX, ERR_SINGULAR, ERR_NONFINITE = 1, 2, 3, 4
ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = 5, 6, 7, 8

F64, F32, BF16 = 0, 1, 2
TOPT_COLUMN, TOPT_MATRIX, TOPT_NONE = 0, 1, 2
U, V = 0, 1
DENSE_ROWMAJOR, CSC, CSR = 0, 1, 2
OPT_USE_GRAPH, OPT_PROFILE, OPT_WAIT_LIMIT = 0, 1, 2
OPT_SPMM_TUNE, OPT_SPMM_SPLIT, OPT_SPMM_CARVEOUT, OPT_SPMM_MASK = 3, 4, 5, 6
OPT_REFINE = 8


class EspnmfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("vdtype", ctypes.c_int),
                ("on_device", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """The library this process loads: the checked build when the
    environment sets ESPNMF_CHECKED=1, else the regular one."""
    return _build.LIB_CHECKED if os.environ.get("ESPNMF_CHECKED") == "1" else _build.LIB


def load():
    """Loads the built library (never builds it)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        st = ctypes.c_int
        sig = {
            "espnmf_init": [ctypes.POINTER(P), ctypes.POINTER(_CSR), i32, i64, i64, st, st,
                            P, st, i32, P],
            "espnmf_destroy": [P],
            "espnmf_als_update_V": [P],
            "espnmf_als_update_U": [P],
            "espnmf_iterate": [P, i32, P, P],
            "espnmf_enforce_topt": [P, st, i64],
            "espnmf_set_factor": [P, st, P, st, i32],
            "espnmf_residual": [P, ctypes.POINTER(d)],
            "espnmf_error": [P, ctypes.POINTER(d)],
            "espnmf_factor_nnz": [P, st, ctypes.POINTER(i64)],
            "espnmf_get_factor": [P, st, st, P, P, P, st, i32],
            "espnmf_set_option": [P, st, i64],
            "espnmf_kernel_stat_count": [P, ctypes.POINTER(i32)],
            "espnmf_kernel_stat": [P, i32, ctypes.POINTER(ctypes.c_char_p),
                                   ctypes.POINTER(i64), ctypes.POINTER(d), ctypes.POINTER(d)],
            "espnmf_kernel_stats_reset": [P],
            "espnmf_launches_per_sweep": [P, ctypes.POINTER(i32)],
            "espnmf_sync": [P],
            "espnmf_checked_flags": [P],
            "espnmf_enforce_topt_buffer": [P, i64, i32, i64, st, i64, st, P],
            "espnmf_enforce_topt_buffer_noalloc": [P, i64, i32, i64, st, i64, st, P],
            "espnmf_loss": [P, ctypes.POINTER(d)],
            "espnmf_grad": [P, st, P, st, i32],
            "espnmf_pg_step": [P, st, d, ctypes.POINTER(d)],
            "espnmf_batch_init": [ctypes.POINTER(P), i32, P, P, P, P, st, st, P, st, i32, i32],
            "espnmf_batch_destroy": [P],
            "espnmf_batch_ctx": [P, i32, ctypes.POINTER(P)],
            "espnmf_batch_set_option": [P, st, i64],
            "espnmf_batch_iterate": [P, i32, P, P, P],
            "espnmf_spmm_config": [P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)],
            "espnmf_spmm_frequent": [P, i32, ctypes.POINTER(i32), ctypes.POINTER(i64)],
            "espnmf_save": [P, ctypes.c_char_p, ctypes.c_uint64],
            "espnmf_solve_gram": [P, i64, i32, i64, P, P, i64, i32, P],
            "espnmf_topic_accuracy": [P, st, P, i32, i32, P],
            "espnmf_load": [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i64)],
            "espnmf_sweeps_done": [P, ctypes.POINTER(i64)],
            "espnmf_select_stats": [P, ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "espnmf_sequential": [ctypes.POINTER(_CSR), i32, i32, i64, i64, i32, st, P, st, i32, P, P,
                                  P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.espnmf_last_error.argtypes = [P]
        lib.espnmf_last_error.restype = ctypes.c_char_p
        lib.espnmf_status_string.argtypes = [ctypes.c_int]
        lib.espnmf_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def exported_symbols():
    """Names the binding resolves in the library (all must exist)."""
    lib = load()
    names = ["espnmf_init", "espnmf_destroy", "espnmf_last_error", "espnmf_status_string",
             "espnmf_als_update_V", "espnmf_als_update_U", "espnmf_iterate",
             "espnmf_enforce_topt", "espnmf_set_factor", "espnmf_residual", "espnmf_error",
             "espnmf_factor_nnz", "espnmf_get_factor", "espnmf_set_option",
             "espnmf_kernel_stat_count", "espnmf_kernel_stat", "espnmf_kernel_stats_reset",
             "espnmf_launches_per_sweep", "espnmf_sync", "espnmf_checked_flags",
             "espnmf_enforce_topt_buffer",
             "espnmf_enforce_topt_buffer_noalloc", "espnmf_loss", "espnmf_grad",
             "espnmf_pg_step", "espnmf_batch_init", "espnmf_batch_destroy",
             "espnmf_batch_ctx", "espnmf_batch_set_option", "espnmf_batch_iterate",
             "espnmf_spmm_config", "espnmf_spmm_frequent", "espnmf_select_stats",
             "espnmf_sequential", "espnmf_save", "espnmf_load", "espnmf_sweeps_done",
             "espnmf_solve_gram", "espnmf_topic_accuracy"]
    return {n: hasattr(lib, n) for n in names}


def _check(st: int, handle=None):
    if st != OK:
        msg = load().espnmf_last_error(handle)
        raise EspnmfError(st, (msg or b"").decode(errors="replace"))


# --- array marshalling ---------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device, keepalive) of a contiguous numpy array / torch tensor."""
    if _is_torch(x):
        if not x.is_contiguous():
            x = x.contiguous()
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x)
    return ctypes.c_void_p(a.ctypes.data), 0, a


def _dtype_code(x) -> int:
    name = str(x.dtype)
    if "bfloat16" in name:
        return BF16
    if "float64" in name:
        return F64
    if "float32" in name:
        return F32
    raise TypeError(f"unsupported element type {x.dtype}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns an espnmf_ctx handle; freed by espnmf_destroy."""

    def __init__(self, handle, n, m, k, compute):
        self.handle = handle
        self.n, self.m, self.k, self.compute = n, m, k, compute

    def __del__(self):
        try:
            if self.handle and getattr(self, "_owned", True):
                load().espnmf_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


# --- the ABI, by name -------------------------------------------------------------

def espnmf_init(rowptr, colidx, values, n: int, m: int, k: int, t_u: int, t_v: int,
                mode: int = TOPT_COLUMN, compute: int = F32, U0=None, stream=None) -> Context:
    lib = load()
    rp, d1, k1 = _ptr(rowptr)
    ci, d2, k2 = _ptr(colidx)
    va, d3, k3 = _ptr(values)
    if not (d1 == d2 == d3):
        raise ValueError("rowptr, colidx and values must all be host or all device arrays")
    if str(rowptr.dtype).split(".")[-1] != "int64" or str(colidx.dtype).split(".")[-1] != "int32":
        raise TypeError("rowptr must be int64 and colidx int32")
    csr = _CSR(int(n), int(m), int(len(colidx)), rp, ci, va, _dtype_code(values), d1)
    up, ud, uk = _ptr(U0)
    h = ctypes.c_void_p()
    st = lib.espnmf_init(ctypes.byref(h), ctypes.byref(csr), int(k), int(t_u), int(t_v),
                         int(mode), int(compute), up, _dtype_code(U0), ud,
                         _stream_handle(stream))
    _check(st, None)
    return Context(h, int(n), int(m), int(k), int(compute))


def espnmf_sequential(rowptr, colidx, values, n: int, m: int, k: int, t_u: int, t_v: int,
                      iters: int, U0, compute: int = F32, stream=None, k2: int = 1,
                      return_seconds: bool = False):
    """Alg. 3 (sequential ALS): k topics found k2 at a time from the initial
    guess U0 (n x k2, or an n-vector for k2 = 1); returns (U, V) as CUDA
    tensors of the compute dtype (n x k, m x k), and with ``return_seconds``
    also the stream time of the iterations (set-up excluded)."""
    import torch
    lib = load()
    rp, d1, _ = _ptr(rowptr)
    ci, d2, _ = _ptr(colidx)
    va, d3, _ = _ptr(values)
    if not (d1 == d2 == d3):
        raise ValueError("rowptr, colidx and values must all be host or all device arrays")
    if tuple(U0.shape) not in ((int(n), int(k2)),) + (((int(n),),) if k2 == 1 else ()):
        raise ValueError(f"U0 must be n x k2 = {n} x {k2}, got {tuple(U0.shape)}")
    csr = _CSR(int(n), int(m), int(len(colidx)), rp, ci, va, _dtype_code(values), d1)
    up, ud, _ = _ptr(U0)
    tdt = torch.float64 if compute == F64 else torch.float32
    # written in full by the library, on its stream, before it returns
    U = torch.empty((int(n), int(k)), dtype=tdt, device="cuda")
    V = torch.empty((int(m), int(k)), dtype=tdt, device="cuda")
    secs = ctypes.c_double()
    _check(lib.espnmf_sequential(ctypes.byref(csr), int(k), int(k2), int(t_u), int(t_v),
                                 int(iters), int(compute), up, _dtype_code(U0), ud,
                                 ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                 ctypes.byref(secs), _stream_handle(stream)))
    return (U, V, secs.value) if return_seconds else (U, V)


def espnmf_destroy(ctx: Context):
    if not getattr(ctx, "_owned", True):
        raise ValueError("a batch problem's context is destroyed with its batch")
    if ctx.handle:
        _check(load().espnmf_destroy(ctx.handle))
        ctx.handle = None


def espnmf_als_update_V(ctx: Context):
    _check(load().espnmf_als_update_V(ctx.handle), ctx.handle)


def espnmf_als_update_U(ctx: Context):
    _check(load().espnmf_als_update_U(ctx.handle), ctx.handle)


def espnmf_iterate(ctx: Context, iters: int, want_measures: bool = True):
    """Runs `iters` sweeps; returns (R, E) numpy arrays (or None)."""
    if want_measures:
        R = np.zeros(max(iters, 1))
        E = np.zeros(max(iters, 1))
        _check(load().espnmf_iterate(ctx.handle, int(iters), R.ctypes.data_as(ctypes.c_void_p),
                                     E.ctypes.data_as(ctypes.c_void_p)), ctx.handle)
        return R[:iters], E[:iters]
    _check(load().espnmf_iterate(ctx.handle, int(iters), None, None), ctx.handle)
    return None


def espnmf_enforce_topt(ctx: Context, which: int, t: int):
    _check(load().espnmf_enforce_topt(ctx.handle, int(which), int(t)), ctx.handle)


def espnmf_set_factor(ctx: Context, which: int, F):
    p, dev, keep = _ptr(F)
    _check(load().espnmf_set_factor(ctx.handle, int(which), p, _dtype_code(F), dev), ctx.handle)


def espnmf_residual(ctx: Context) -> float:
    r = ctypes.c_double()
    _check(load().espnmf_residual(ctx.handle, ctypes.byref(r)), ctx.handle)
    return r.value


def espnmf_error(ctx: Context) -> float:
    e = ctypes.c_double()
    _check(load().espnmf_error(ctx.handle, ctypes.byref(e)), ctx.handle)
    return e.value


def espnmf_loss(ctx: Context) -> float:
    """f = ||A - U V^T||_F^2 at the current U, V (FP64 identity on the device)."""
    f = ctypes.c_double()
    _check(load().espnmf_loss(ctx.handle, ctypes.byref(f)), ctx.handle)
    return f.value


def espnmf_grad(ctx: Context, which: int, out=None, dtype=np.float64):
    """Dense gradient of f with respect to U (which=U) or V (which=V).

    ``out`` may be a contiguous rows x k float32/float64 numpy array or torch
    tensor (host or CUDA); by default a new numpy array of ``dtype``.  For a
    CUDA ``out`` the call synchronises the context's stream before it returns.
    """
    rows = ctx.n if which == U else ctx.m
    if out is None:
        out = np.zeros((rows, ctx.k), dtype=dtype)
    if tuple(out.shape) != (rows, ctx.k):
        raise ValueError(f"out must be {rows} x {ctx.k}")
    if _is_torch(out) and not out.is_contiguous():
        raise ValueError("out must be contiguous")
    p, dev, keep = _ptr(out)
    if not _is_torch(out) and keep is not out:
        raise ValueError("out must be a contiguous numpy array")
    lib = load()
    _check(lib.espnmf_grad(ctx.handle, int(which), p, _dtype_code(out), dev), ctx.handle)
    if dev:
        _check(lib.espnmf_sync(ctx.handle), ctx.handle)
    return out


def espnmf_pg_step(ctx: Context, which: int, eta: float = 0.0) -> float:
    """One projected-gradient step on the factor's support; returns the step
    used (eta <= 0: 1 / (2 lambda_max) of the other factor's Gram)."""
    e = ctypes.c_double()
    _check(load().espnmf_pg_step(ctx.handle, int(which), float(eta), ctypes.byref(e)),
           ctx.handle)
    return e.value


def espnmf_factor_nnz(ctx: Context, which: int) -> int:
    z = ctypes.c_int64()
    _check(load().espnmf_factor_nnz(ctx.handle, int(which), ctypes.byref(z)), ctx.handle)
    return z.value


def espnmf_get_factor(ctx: Context, which: int, layout: int = DENSE_ROWMAJOR,
                      dtype=np.float64):
    """Returns the factor as numpy: a dense rows x k array, or (ptr, idx, val)."""
    rows = ctx.n if which == U else ctx.m
    code = F64 if np.dtype(dtype) == np.float64 else F32
    lib = load()
    if layout == DENSE_ROWMAJOR:
        out = np.zeros((rows, ctx.k), dtype=dtype)
        _check(lib.espnmf_get_factor(ctx.handle, int(which), layout, None, None,
                                     out.ctypes.data_as(ctypes.c_void_p), code, 0), ctx.handle)
        return out
    nnz = espnmf_factor_nnz(ctx, which)
    nptr = ctx.k + 1 if layout == CSC else rows + 1
    ptr = np.zeros(nptr, dtype=np.int64)
    idx = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros(max(nnz, 1), dtype=dtype)
    _check(lib.espnmf_get_factor(ctx.handle, int(which), layout,
                                 ptr.ctypes.data_as(ctypes.c_void_p),
                                 idx.ctypes.data_as(ctypes.c_void_p),
                                 val.ctypes.data_as(ctypes.c_void_p), code, 0), ctx.handle)
    return ptr, idx[:nnz], val[:nnz]


def espnmf_spmm_config(ctx: Context, product: int):
    """(split, carveout, mask) of product 0 (A V) or 1 (A^T U)."""
    g, c, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().espnmf_spmm_config(ctx.handle, int(product), ctypes.byref(g), ctypes.byref(c),
                                     ctypes.byref(m)), ctx.handle)
    return g.value, c.value, m.value


def espnmf_solve_gram(Y, G, refine: bool = False, stream=None):
    """X = Y G^-1 (unprojected) for a CUDA float32 Y (rows x k) and a CUDA
    float64 G (k x k), with one refinement step when ``refine``."""
    import torch
    rows, k = Y.shape
    Gc = G.contiguous()
    X = torch.empty((rows, k), dtype=torch.float32, device=Y.device)
    st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(load().espnmf_solve_gram(ctypes.c_void_p(Y.data_ptr()), rows, k, Y.stride(0),
                                    ctypes.c_void_p(Gc.data_ptr()),
                                    ctypes.c_void_p(X.data_ptr()), k, int(bool(refine)),
                                    ctypes.c_void_p(st)))
    return X


def espnmf_topic_accuracy(ctx: Context, labels, n_classes: int, which: int = V) -> np.ndarray:
    """Eq. 3-4 accuracy of each column of the factor (default V) against
    integer class labels (numpy or CUDA int32 tensor, one per row)."""
    acc = np.zeros(ctx.k, dtype=np.float64)
    if _is_torch(labels) and labels.is_cuda:
        lab, dev = labels.to(dtype=__import__("torch").int32).contiguous(), 1
        ptr = ctypes.c_void_p(lab.data_ptr())
    else:
        lab, dev = np.ascontiguousarray(labels, dtype=np.int32), 0
        ptr = lab.ctypes.data_as(ctypes.c_void_p)
    _check(load().espnmf_topic_accuracy(ctx.handle, int(which), ptr, int(n_classes), dev,
                                        acc.ctypes.data_as(ctypes.c_void_p)), ctx.handle)
    return acc


def espnmf_save(ctx: Context, path: str, tag: int = 0):
    """Writes the context's state (U, V, their Grams, the sweep count and
    ``tag``) to ``path``."""
    _check(load().espnmf_save(ctx.handle, os.fsencode(path), int(tag)), ctx.handle)


def espnmf_load(ctx: Context, path: str):
    """Restores a saved state into ``ctx``; returns (tag, sweeps)."""
    tag, sw = ctypes.c_uint64(), ctypes.c_int64()
    _check(load().espnmf_load(ctx.handle, os.fsencode(path), ctypes.byref(tag), ctypes.byref(sw)),
           ctx.handle)
    return tag.value, sw.value


def espnmf_sweeps_done(ctx: Context) -> int:
    sw = ctypes.c_int64()
    _check(load().espnmf_sweeps_done(ctx.handle, ctypes.byref(sw)), ctx.handle)
    return sw.value


def espnmf_select_stats(ctx: Context):
    """(warm, full): column selections that started from the previous
    threshold and found the new one near it, and those searched from scratch."""
    w, f = ctypes.c_int64(), ctypes.c_int64()
    _check(load().espnmf_select_stats(ctx.handle, ctypes.byref(w), ctypes.byref(f)), ctx.handle)
    return w.value, f.value


def espnmf_spmm_frequent(ctx: Context, product: int):
    """(h, hnnz) of the frequent part of product 0 (A V) or 1 (A^T U)."""
    h, e = ctypes.c_int32(), ctypes.c_int64()
    _check(load().espnmf_spmm_frequent(ctx.handle, int(product), ctypes.byref(h), ctypes.byref(e)),
           ctx.handle)
    return h.value, e.value


def espnmf_set_option(ctx: Context, opt: int, value: int):
    _check(load().espnmf_set_option(ctx.handle, int(opt), int(value)), ctx.handle)


def espnmf_kernel_stats(ctx: Context):
    """{name: (launches, total_ms, bytes)} of the profiled kernel launches."""
    lib = load()
    n = ctypes.c_int32()
    _check(lib.espnmf_kernel_stat_count(ctx.handle, ctypes.byref(n)), ctx.handle)
    out = {}
    for i in range(n.value):
        name = ctypes.c_char_p()
        cnt = ctypes.c_int64()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        _check(lib.espnmf_kernel_stat(ctx.handle, i, ctypes.byref(name), ctypes.byref(cnt),
                                      ctypes.byref(ms), ctypes.byref(by)), ctx.handle)
        out[name.value.decode()] = (cnt.value, ms.value, by.value)
    return out


def espnmf_kernel_stats_reset(ctx: Context):
    _check(load().espnmf_kernel_stats_reset(ctx.handle), ctx.handle)


def espnmf_launches_per_sweep(ctx: Context) -> int:
    c = ctypes.c_int32()
    _check(load().espnmf_launches_per_sweep(ctx.handle, ctypes.byref(c)), ctx.handle)
    return c.value


def espnmf_sync(ctx: Context):
    _check(load().espnmf_sync(ctx.handle), ctx.handle)


def espnmf_checked_flags() -> int:
    """The bounds checks that failed since the last call (checked build;
    raises EspnmfError(UNSUPPORTED) in the regular build)."""
    f = ctypes.c_uint32()
    _check(load().espnmf_checked_flags(ctypes.byref(f)))
    return f.value


def espnmf_enforce_topt_buffer(X, t: int, mode: int = TOPT_COLUMN, stream=None):
    """In-place projection + top-t on a CUDA tensor X (rows x k, row-major)."""
    if not (_is_torch(X) and X.is_cuda):
        raise TypeError("X must be a CUDA tensor")
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be 2-D with unit column stride")
    _check(load().espnmf_enforce_topt_buffer(ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                             X.shape[1], X.stride(0), _dtype_code(X), int(t),
                                             int(mode), _stream_handle(stream)))


NOALLOC_MAX_ELEMS = 262144


def espnmf_enforce_topt_buffer_noalloc(X, t: int, mode: int = TOPT_COLUMN, stream=None):
    """espnmf_enforce_topt_buffer without any device allocation (scratch in
    a fixed array inside the library; see include/espnmf.h for the size
    limit and the rules on concurrent calls)."""
    if not (_is_torch(X) and X.is_cuda):
        raise TypeError("X must be a CUDA tensor")
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be 2-D with unit column stride")
    _check(load().espnmf_enforce_topt_buffer_noalloc(ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                                     X.shape[1], X.stride(0), _dtype_code(X),
                                                     int(t), int(mode), _stream_handle(stream)))


# --- batched problems --------------------------------------------------------------

class Batch:
    """Owns an espnmf_batch handle (and, through it, one context per problem)."""

    def __init__(self, handle, shapes, compute, keep):
        self.handle = handle
        self.shapes = shapes          # [(n, m, k)]
        self.compute = compute
        self._keep = keep

    def __len__(self):
        return len(self.shapes)

    def ctx(self, i: int) -> Context:
        """Problem i's context (owned by the batch: not destroyed by the view)."""
        h = ctypes.c_void_p()
        _check(load().espnmf_batch_ctx(self.handle, int(i), ctypes.byref(h)))
        n, m, k = self.shapes[i]
        view = Context.__new__(Context)
        view.handle, view.n, view.m, view.k, view.compute = h, n, m, k, self.compute
        view._owned = False
        view._batch = self
        return view

    def __del__(self):
        try:
            if self.handle:
                load().espnmf_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def espnmf_batch_init(problems, mode: int = TOPT_COLUMN, compute: int = F32,
                      streams: int = 0) -> Batch:
    """problems: a list of (rowptr, colidx, values, n, m, k, t_u, t_v, U0);
    arrays as for espnmf_init, all on the host or all on the device."""
    count = len(problems)
    csrs = (_CSR * count)()
    ks = (ctypes.c_int32 * count)()
    tus = (ctypes.c_int64 * count)()
    tvs = (ctypes.c_int64 * count)()
    u0s = (ctypes.c_void_p * count)()
    keep, shapes = [], []
    u0_dev, u0_dtype = None, None
    for i, (rowptr, colidx, values, n, m, k, t_u, t_v, U0) in enumerate(problems):
        rp, rdev, rk = _ptr(rowptr)
        ci, _, ck = _ptr(colidx)
        va, _, vk = _ptr(values)
        up, udev, uk = _ptr(U0)
        keep += [rk, ck, vk, uk]
        csrs[i] = _CSR(n, m, int(len(colidx)), rp, ci, va, _dtype_code(values), rdev)
        ks[i], tus[i], tvs[i] = k, t_u, t_v
        u0s[i] = up
        if u0_dev is None:
            u0_dev, u0_dtype = udev, _dtype_code(U0)
        elif (udev, _dtype_code(U0)) != (u0_dev, u0_dtype):
            raise ValueError("all U0 must share one dtype and one location")
        shapes.append((n, m, k))
    h = ctypes.c_void_p()
    _check(load().espnmf_batch_init(ctypes.byref(h), count, csrs, ks, tus, tvs, int(mode),
                                    int(compute), u0s, u0_dtype, u0_dev, int(streams)))
    return Batch(h, shapes, compute, None)


def espnmf_batch_set_option(b: Batch, opt: int, value: int):
    _check(load().espnmf_batch_set_option(b.handle, int(opt), int(value)))


def espnmf_batch_iterate(b: Batch, iters: int, want_measures: bool = True):
    """Returns (status array, R [nprob x iters] or None, E or None); raises
    only for failures of the batch itself (per-problem failures are in the
    status array)."""
    count = len(b)
    status = np.zeros(count, dtype=np.int32)
    R = np.zeros((count, max(iters, 1))) if want_measures else None
    E = np.zeros((count, max(iters, 1))) if want_measures else None
    st = load().espnmf_batch_iterate(
        b.handle, int(iters), status.ctypes.data_as(ctypes.c_void_p),
        R.ctypes.data_as(ctypes.c_void_p) if want_measures else None,
        E.ctypes.data_as(ctypes.c_void_p) if want_measures else None)
    if st != OK and not status.any():
        _check(st)
    if want_measures:
        R, E = R[:, :iters], E[:, :iters]
    return status, R, E
