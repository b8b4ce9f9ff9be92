"""FP64 CPU oracle for enforced-sparsity ALS NMF (arXiv:1510.05237).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product never imports
this package; the oracle shares no code with the CUDA path.

``espnmf_oracle.c`` holds the arithmetic (plain C, FP64, single-threaded);
this module compiles it with gcc on first use and wraps it with ctypes.
Matrices come in as ``gen.Corpus`` (CSR over terms) and dense row-major
float64 factors.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "espnmf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_LIB_OMP = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

OK, INVALID_ARG, BAD_MATRIX, SINGULAR, NONFINITE, OOM = 0, 1, 2, 3, 4, 5
COLUMN, MATRIX, NONE = 0, 1, 2


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def build(force: bool = False, threads: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``, or with
    ``threads`` the same source with OpenMP into ``liboracle_omp.so`` (used
    only for the benchmark's all-cores CPU baseline; its results are
    bitwise those of the single-threaded build)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    lib = _LIB_OMP if threads else _LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", *(["-fopenmp"] if threads else []),
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, lib)
    return lib


def _load(threads: bool = False):
    with _lock:
        if threads in _libs:
            return _libs[threads]
        lib = ctypes.CDLL(build(threads=threads))
        i64, i32, d = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        P = ctypes.c_void_p
        csr = [i64, i64, P, P, P, i32]
        sig = {
            "or_spmm_At": (None, csr + [P, P]),
            "or_spmm_A": (None, csr + [P, P]),
            "or_gram": (None, [i64, i32, P, P]),
            "or_cholesky": (ctypes.c_int, [i32, P, P, P]),
            "or_ls_solve": (ctypes.c_int, [i64, i32, P, P, P]),
            "or_project": (ctypes.c_int, [P, i64]),
            "or_topt": (ctypes.c_int, [P, i64, i32, i64, ctypes.c_int]),
            "or_update_V": (ctypes.c_int, csr + [P, i64, ctypes.c_int, P, P]),
            "or_update_U": (ctypes.c_int, csr + [P, i64, ctypes.c_int, P, P]),
            "or_residual": (d, [i64, i32, P, P]),
            "or_norm2_A": (d, [i64, P]),
            "or_loss": (d, csr + [P, P]),
            "or_error_identity": (d, csr + [P, P]),
            "or_error_direct": (d, csr + [P, P]),
            "or_iterate": (ctypes.c_int, csr + [P, i64, i64, ctypes.c_int, i32,
                                               P, P, P, P]),
            "or_grad_U": (None, csr + [P, P, P]),
            "or_grad_V": (None, csr + [P, P, P]),
            "or_lambda_max": (d, [i32, P]),
            "or_pg_step": (ctypes.c_int, csr + [P, P, ctypes.c_int]),
            "or_topic_accuracy": (ctypes.c_int, [i64, i32, P, P, i32, P]),
            "or_sequential": (ctypes.c_int, csr[:5] + [i32, i32, P, i64, i64, i32, P, P, P, P]),
            "or_set_threads": (None, [i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _libs[threads] = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _CSR:
    """Keeps contiguous copies alive for the duration of a call."""

    def __init__(self, A):
        self.n, self.m = int(A.n), int(A.m)
        self.rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        self.colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
        self.val = _f64(A.val)

    def args(self, k: int):
        return [self.n, self.m, _ptr(self.rowptr), _ptr(self.colidx),
                _ptr(self.val), int(k)]


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(st, what)


# --------------------------------------------------------------------------
# Building blocks

def spmm_At(A, U: np.ndarray) -> np.ndarray:
    """A^T U (m x k)."""
    U = _f64(U)
    k = U.shape[1]
    B = np.zeros((A.m, k))
    _load().or_spmm_At(*_CSR(A).args(k), _ptr(U), _ptr(B))
    return B


def spmm_A(A, V: np.ndarray) -> np.ndarray:
    """A V (n x k)."""
    V = _f64(V)
    k = V.shape[1]
    B = np.zeros((A.n, k))
    _load().or_spmm_A(*_CSR(A).args(k), _ptr(V), _ptr(B))
    return B


def gram(F: np.ndarray) -> np.ndarray:
    F = _f64(F)
    G = np.zeros((F.shape[1], F.shape[1]))
    _load().or_gram(F.shape[0], F.shape[1], _ptr(F), _ptr(G))
    return G


def cholesky(G: np.ndarray):
    """(L, active) of the reduced Cholesky factorisation."""
    G = _f64(G)
    k = G.shape[0]
    L = np.zeros((k, k))
    act = np.zeros(k, dtype=np.int32)
    _check(_load().or_cholesky(k, _ptr(G), _ptr(L), _ptr(act)), "cholesky")
    return L, act.astype(bool)


def ls_solve(B: np.ndarray, G: np.ndarray) -> np.ndarray:
    """X with X G = B, row by row."""
    B, G = _f64(B), _f64(G)
    X = np.zeros_like(B)
    _check(_load().or_ls_solve(B.shape[0], B.shape[1], _ptr(B), _ptr(G), _ptr(X)),
           "ls_solve")
    return X


def project(X: np.ndarray) -> np.ndarray:
    X = _f64(X).copy()
    _check(_load().or_project(_ptr(X), X.size), "project")
    return X


def topt(X: np.ndarray, t: int, mode: int = COLUMN) -> np.ndarray:
    """Keep the t largest positive entries (per column or overall)."""
    X = _f64(X).copy()
    _check(_load().or_topt(_ptr(X), X.shape[0], X.shape[1], int(t), int(mode)), "topt")
    return X


# --------------------------------------------------------------------------
# Alg. 2 half-steps, measures and the sweep loop

def update_V(A, U: np.ndarray, t_v: int, mode: int = COLUMN,
             return_pre: bool = False):
    U = _f64(U)
    k = U.shape[1]
    V = np.zeros((A.m, k))
    pre = np.zeros((A.m, k))
    _check(_load().or_update_V(*_CSR(A).args(k), _ptr(U), int(t_v), int(mode),
                               _ptr(V), _ptr(pre)), "update_V")
    return (V, pre) if return_pre else V


def update_U(A, V: np.ndarray, t_u: int, mode: int = COLUMN,
             return_pre: bool = False):
    V = _f64(V)
    k = V.shape[1]
    U = np.zeros((A.n, k))
    pre = np.zeros((A.n, k))
    _check(_load().or_update_U(*_CSR(A).args(k), _ptr(V), int(t_u), int(mode),
                               _ptr(U), _ptr(pre)), "update_U")
    return (U, pre) if return_pre else U


def residual(Unew: np.ndarray, Uold: np.ndarray) -> float:
    Unew, Uold = _f64(Unew), _f64(Uold)
    return _load().or_residual(Unew.shape[0], Unew.shape[1], _ptr(Unew), _ptr(Uold))


def norm2_A(A) -> float:
    v = _f64(A.val)
    return _load().or_norm2_A(len(v), _ptr(v))


def loss(A, U, V) -> float:
    U, V = _f64(U), _f64(V)
    return _load().or_loss(*_CSR(A).args(U.shape[1]), _ptr(U), _ptr(V))


def error_identity(A, U, V) -> float:
    U, V = _f64(U), _f64(V)
    return _load().or_error_identity(*_CSR(A).args(U.shape[1]), _ptr(U), _ptr(V))


def error_direct(A, U, V) -> float:
    U, V = _f64(U), _f64(V)
    return _load().or_error_direct(*_CSR(A).args(U.shape[1]), _ptr(U), _ptr(V))


def iterate(A, U0: np.ndarray, t_u: int, t_v: int, mode: int = COLUMN,
            iters: int = 1, threads: int | None = None):
    """Alg. 2 for ``iters`` sweeps.  Returns (U, V, R[iters], E[iters]).
    With ``threads``, the OpenMP build on that many threads (same results)."""
    lib = _load(True) if threads else _load()
    if threads:
        lib.or_set_threads(int(threads))
    U0 = _f64(U0)
    k = U0.shape[1]
    U = np.zeros((A.n, k))
    V = np.zeros((A.m, k))
    R = np.zeros(max(iters, 1))
    E = np.zeros(max(iters, 1))
    _check(lib.or_iterate(*_CSR(A).args(k), _ptr(U0), int(t_u), int(t_v),
                              int(mode), int(iters), _ptr(R), _ptr(E), _ptr(U),
                              _ptr(V)), "iterate")
    return U, V, R[:iters], E[:iters]


def grad_U(A, U, V) -> np.ndarray:
    U, V = _f64(U), _f64(V)
    g = np.zeros_like(U)
    _load().or_grad_U(*_CSR(A).args(U.shape[1]), _ptr(U), _ptr(V), _ptr(g))
    return g


def grad_V(A, U, V) -> np.ndarray:
    U, V = _f64(U), _f64(V)
    g = np.zeros_like(V)
    _load().or_grad_V(*_CSR(A).args(U.shape[1]), _ptr(U), _ptr(V), _ptr(g))
    return g


def lambda_max(G: np.ndarray) -> float:
    G = _f64(G)
    return _load().or_lambda_max(G.shape[0], _ptr(G))


def pg_step(A, U, V, which: int):
    """One projected-gradient polish step of U (which=0) or V (which=1)."""
    U, V = _f64(U).copy(), _f64(V).copy()
    _check(_load().or_pg_step(*_CSR(A).args(U.shape[1]), _ptr(U), _ptr(V),
                              int(which)), "pg_step")
    return U, V


def topic_accuracy(V: np.ndarray, labels: np.ndarray, n_J: int) -> np.ndarray:
    """Sec. 3.2, Eq. 3-4: clustering accuracy of each column of V (documents
    belong to a topic where V is nonzero), same-label pairs counted one by
    one.  Returns acc[k]."""
    V = _f64(V)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    acc = np.zeros(V.shape[1])
    _check(_load().or_topic_accuracy(V.shape[0], V.shape[1], _ptr(V), _ptr(lab), int(n_J),
                                     _ptr(acc)), "topic_accuracy")
    return acc


def sequential(A, U0: np.ndarray, k: int, t_u: int, t_v: int, iters: int,
               return_pre: bool = False, k2: int = 1):
    """Sec. 4, Alg. 3: k topics found k2 at a time (k a multiple of k2), each
    block from the same initial guess U0 (n x k2; an n-vector when k2 = 1),
    ``iters`` sweeps per block; the first block is Alg. 2.  Returns (U, V),
    and with ``return_pre`` also the last block's last V2 and U2 before the
    projection (m x k2, n x k2; vectors when k2 = 1)."""
    U0 = _f64(np.asarray(U0).reshape(A.n, k2))
    U = np.zeros((A.n, k))
    V = np.zeros((A.m, k))
    vpre = np.zeros((A.m, k2))
    upre = np.zeros((A.n, k2))
    c = _CSR(A)
    _check(_load().or_sequential(*c.args(1)[:5], int(k), int(k2), _ptr(U0), int(t_u), int(t_v),
                                 int(iters), _ptr(U), _ptr(V), _ptr(vpre), _ptr(upre)),
           "sequential")
    if k2 == 1:
        vpre, upre = vpre[:, 0], upre[:, 0]
    return (U, V, vpre, upre) if return_pre else (U, V)
