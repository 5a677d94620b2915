"""Explicit basis and CSR Hamiltonian of the oracle (ctypes front end of basis.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Pinned by: the worked example L=4, N=2 of Sec. 2 (tests/golden/basis_L4_N2.txt), the
sector dimensions printed in Table I and Sec. 5 (tests/golden/dimensions.txt), brute-force
enumeration of all 2^L integers, and a Kronecker-product construction of Eq. 1 in the
full 2^L space (oracle.dense) for every L <= 10.  orc_moments (basis.c) is the engine of
oracle.moments and is pinned there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "basis.c")


def build(force: bool = False) -> str:
    """Compile basis.c into oracle/lib/liboracle.so with gcc (plain C, no target flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, u64p, dp, i64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64), \
            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
        L.orc_binom.restype = i64
        L.orc_binom.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_basis.restype = i64
        L.orc_basis.argtypes = [ctypes.c_int, ctypes.c_int, u64p, i64]
        L.orc_lookup.restype = i64
        L.orc_lookup.argtypes = [u64p, i64, ctypes.c_uint64]
        L.orc_ham_nnz.restype = i64
        L.orc_ham_nnz.argtypes = [ctypes.c_int, u64p, i64, ctypes.c_int]
        L.orc_diag.restype = ctypes.c_double
        L.orc_diag.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               dp, ctypes.c_int]
        L.orc_ham_csr.restype = ctypes.c_int
        L.orc_ham_csr.argtypes = [ctypes.c_int, u64p, i64, ctypes.c_double, ctypes.c_double,
                                  dp, ctypes.c_int, i64p, i64p, dp]
        L.orc_spmv.restype = None
        L.orc_spmv.argtypes = [i64, i64p, i64p, dp, dp, dp]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def binom(n: int, k: int) -> int:
    return int(lib().orc_binom(n, k))


def basis(L: int, N: int) -> np.ndarray:
    """Sorted integer basis of the (L, N) sector by Algorithm 2."""
    D = binom(L, N)
    out = np.zeros(D, dtype=np.uint64)
    got = lib().orc_basis(L, N, _p(out, ctypes.c_uint64), D)
    if got != D:
        raise ValueError(f"bad sector L={L} N={N}")
    return out


def lookup(b: np.ndarray, s: int) -> int:
    """Binary lookup of state s in the sorted basis (-1 when absent)."""
    b = np.ascontiguousarray(b, dtype=np.uint64)
    return int(lib().orc_lookup(_p(b, ctypes.c_uint64), b.size, ctypes.c_uint64(s)))


class CSR:
    """Real symmetric sector Hamiltonian of Eq. 1 (XXZ form) in CSR storage."""

    def __init__(self, L, N, J, Delta, h, pbc=True, b=None):
        self.L, self.N = L, N
        self.basis = basis(L, N) if b is None else b
        D = self.basis.size
        h = np.ascontiguousarray(h, dtype=np.float64)
        assert h.size == L
        l = lib()
        nnz = l.orc_ham_nnz(L, _p(self.basis, ctypes.c_uint64), D, int(pbc))
        self.rowptr = np.zeros(D + 1, dtype=np.int64)
        self.col = np.zeros(nnz, dtype=np.int64)
        self.val = np.zeros(nnz, dtype=np.float64)
        rc = l.orc_ham_csr(L, _p(self.basis, ctypes.c_uint64), D, float(J), float(Delta),
                           _p(h, ctypes.c_double), int(pbc), _p(self.rowptr, ctypes.c_int64),
                           _p(self.col, ctypes.c_int64), _p(self.val, ctypes.c_double))
        if rc != 0:
            raise RuntimeError("hopped state not found in basis")
        self.D = D

    def matvec(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.empty_like(x)
        lib().orc_spmv(self.D, _p(self.rowptr, ctypes.c_int64), _p(self.col, ctypes.c_int64),
                       _p(self.val, ctypes.c_double), _p(x.view(np.float64), ctypes.c_double),
                       _p(y.view(np.float64), ctypes.c_double))
        return y

    def norm_inf(self) -> float:
        """Max absolute row sum (an upper bound of the spectral radius)."""
        a = np.abs(self.val)
        return float(np.max(np.add.reduceat(a, self.rowptr[:-1]))) if self.D else 0.0

    def dense(self) -> np.ndarray:
        H = np.zeros((self.D, self.D))
        for r in range(self.D):
            for k in range(self.rowptr[r], self.rowptr[r + 1]):
                H[r, self.col[k]] += self.val[k]
        return H


def row_apply(L, J, Delta, h, pbc, b: np.ndarray, x: np.ndarray, rows) -> np.ndarray:
    """(H x)[r] for the selected rows r only, from the explicit sorted basis b.

    Same construction as CSR (Eq. 1 by bit operations, column by binary lookup), one row
    at a time, for sizes whose full CSR matrix does not fit in host memory.

    Pinned by: CSR.matvec on every row for several (L, N, boundary), and the Kronecker-
    product H of oracle.dense on sampled rows of every sector for L <= 10
    (tests/test_oracle_moments.py).
    """
    l = lib()
    h = np.ascontiguousarray(h, dtype=np.float64)
    bp = _p(b, ctypes.c_uint64)
    bonds = [(i, i + 1) for i in range(L - 1)] + ([(L - 1, 0)] if pbc and L >= 3 else [])
    out = np.zeros(len(rows), dtype=np.complex128)
    for k, r in enumerate(rows):
        s = int(b[r])
        acc = l.orc_diag(ctypes.c_uint64(s), L, float(J), float(Delta), _p(h, ctypes.c_double),
                         int(pbc)) * x[r]
        for (i, j) in bonds:
            if ((s >> i) & 1) != ((s >> j) & 1):
                c = int(l.orc_lookup(bp, b.size, ctypes.c_uint64(s ^ ((1 << i) | (1 << j)))))
                acc += 0.5 * J * x[c]
        out[k] = acc
    return out
