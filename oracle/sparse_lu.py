"""The oracle's sparse direct solver: ctypes binding of oracle/olu.c.

TEST INFRASTRUCTURE ONLY (imported by oracle/ers_oracle.py; only tests/, the smoke check and
the benchmark's CPU baseline import the oracle).  It shares no code with the CUDA library.

olu.c holds a minimum-degree ordering (quotient graph, exact degrees) and a left-looking
sparse LU with threshold partial pivoting (Gilbert & Peierls); see its header.  The C file is
compiled with the host C compiler on first use (or by the package build) into
oracle/_build/libolu.so, which is git-ignored; every machine builds its own.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "olu.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libolu.so")
_lock = threading.Lock()
_lib = None

OLU_OK, OLU_SINGULAR, OLU_NOMEM, OLU_INVALID = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile olu.c into a shared library (plain C99, -O2) unless an up-to-date one exists."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler for the oracle's sparse LU")
    tmp = f"{LIB}.{os.getpid()}.tmp"
    cmd = [cc, "-std=c99", "-O2", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sparse LU build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.olu_order.argtypes = [C.c_int32, P, P, P]
            L.olu_order.restype = C.c_int
            L.olu_factor.argtypes = [C.c_int32, P, P, P, P, C.c_double, C.POINTER(C.c_void_p)]
            L.olu_factor.restype = C.c_int
            L.olu_solve.argtypes = [P, C.c_int32, P, P, P]
            L.olu_solve.restype = None
            L.olu_free.argtypes = [P]
            L.olu_free.restype = None
            L.olu_nnz_l.argtypes = [P]
            L.olu_nnz_l.restype = C.c_int64
            L.olu_nnz_u.argtypes = [P]
            L.olu_nnz_u.restype = C.c_int64
            L.olu_export.argtypes = [P] * 9
            L.olu_export.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def min_degree_order(A) -> np.ndarray:
    """Minimum-degree elimination order of the pattern of A + A^T (new -> old)."""
    A = sp.csc_matrix(A)
    n = A.shape[0]
    ptr = np.ascontiguousarray(A.indptr, np.int32)
    idx = np.ascontiguousarray(A.indices, np.int32)
    perm = np.zeros(n, np.int32)
    rc = lib().olu_order(n, _ptr(ptr), _ptr(idx), _ptr(perm))
    if rc != OLU_OK:
        raise MemoryError("minimum-degree ordering ran out of memory")
    return perm


class SingularMatrixError(ArithmeticError):
    pass


class SparseLU:
    """P A Q = L U of a square sparse matrix: Q from the minimum-degree order of A + A^T,
    P from threshold partial pivoting (the diagonal row is kept while
    |a_diag| >= tau max |a|)."""

    def __init__(self, A, tau: float = 0.1, order: np.ndarray | None = None):
        A = sp.csc_matrix(A, dtype=np.float64)
        A.sort_indices()
        n = A.shape[0]
        if A.shape[1] != n:
            raise ValueError("square matrix expected")
        self.n = n
        self._ptr = np.ascontiguousarray(A.indptr, np.int32)
        self._idx = np.ascontiguousarray(A.indices, np.int32)
        self._val = np.ascontiguousarray(A.data, np.float64)
        self.q = (min_degree_order(A) if order is None
                  else np.ascontiguousarray(order, np.int32))
        self._h = C.c_void_p()
        rc = lib().olu_factor(n, _ptr(self._ptr), _ptr(self._idx), _ptr(self._val),
                              _ptr(self.q), float(tau), C.byref(self._h))
        if rc == OLU_SINGULAR:
            raise SingularMatrixError("matrix is exactly singular")
        if rc != OLU_OK:
            raise RuntimeError(f"oracle sparse LU failed ({rc})")
        self._work = np.zeros(max(n, 1))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().olu_free(h)
            self._h = None

    def solve(self, b) -> np.ndarray:
        """A^{-1} b for a vector (n,) or a column block (n, k)."""
        b = np.asarray(b, dtype=np.float64)
        if b.shape[0] != self.n:
            raise ValueError("right-hand side has the wrong length")
        cols = b.reshape(self.n, -1)
        bt = np.ascontiguousarray(cols.T)               # k x n, one right-hand side per row
        xt = np.empty_like(bt)
        lib().olu_solve(self._h, bt.shape[0], _ptr(bt), _ptr(xt), _ptr(self._work))
        return xt.T.reshape(b.shape)

    @property
    def nnz(self) -> int:
        return int(lib().olu_nnz_l(self._h) + lib().olu_nnz_u(self._h))

    def factors(self):
        """(L, U, prow, q) with (A[prow][:, q]) = L U; L unit lower, U upper (CSC)."""
        L_ = lib()
        n = self.n
        nl = int(L_.olu_nnz_l(self._h)) - n
        nu = int(L_.olu_nnz_u(self._h))
        Lp = np.zeros(n + 1, np.int64); Li = np.zeros(max(nl, 1), np.int32)
        Lx = np.zeros(max(nl, 1)); Up = np.zeros(n + 1, np.int64)
        Ui = np.zeros(max(nu, 1), np.int32); Ux = np.zeros(max(nu, 1))
        prow = np.zeros(n, np.int32); q = np.zeros(n, np.int32)
        L_.olu_export(self._h, _ptr(Lp), _ptr(Li), _ptr(Lx), _ptr(Up), _ptr(Ui), _ptr(Ux),
                      _ptr(prow), _ptr(q))
        Lm = sp.csc_matrix((Lx[:nl], Li[:nl], Lp), shape=(n, n)) + sp.identity(n, format="csc")
        Um = sp.csc_matrix((Ux[:nu], Ui[:nu], Up), shape=(n, n))
        return Lm, Um, prow, q
