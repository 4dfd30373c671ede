"""ctypes binding and build step for the C part of the oracle (be_oracle.c).

TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
benchmark's CPU-baseline leg; never by the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "be_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile be_oracle.c with the host C compiler (portable flags, no -march)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load(path: str):
    """Load a compiled copy of be_oracle.c and declare its signatures."""
    L = ctypes.CDLL(path)
    d = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    L.or_be_tridiag.argtypes = [i64, i64, ctypes.c_double, d, d, d, d, d, d]
    L.or_be_tridiag.restype = ctypes.c_int
    L.or_be_banded.argtypes = [i64, i64, i64, ctypes.c_double, d, d, i64, d, d]
    L.or_be_banded.restype = ctypes.c_int
    L.or_shifted_tridiag_solve.argtypes = [i64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, d, d, d, d, d]
    L.or_shifted_tridiag_solve.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib




def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def be_tridiag(tau, lo, diag, up, G, mdiag=None):
    """Sequential backward Euler for tridiagonal K; G (l, n) -> U (l, n)."""
    G = _c(G)
    nt, n = G.shape
    lo, diag, up = _c(lo), _c(diag), _c(up)
    md = None if mdiag is None else _c(mdiag)
    U = np.empty_like(G)
    rc = lib().or_be_tridiag(n, nt, float(tau), _p(lo), _p(diag), _p(up), _p(md), _p(G), _p(U))
    if rc != 0:
        raise RuntimeError(f"or_be_tridiag failed with code {rc}")
    return U


def be_banded(tau, kl, ku, Kband, G, mdiag=None):
    """Sequential backward Euler for banded K given row-major band storage."""
    G = _c(G)
    nt, n = G.shape
    Kband = _c(Kband)
    assert Kband.shape == (n, kl + ku + 1)
    md = None if mdiag is None else _c(mdiag)
    U = np.empty_like(G)
    rc = lib().or_be_banded(n, kl, ku, float(tau), _p(Kband), _p(md), nt, _p(G), _p(U))
    if rc != 0:
        raise RuntimeError(f"or_be_banded failed with code {rc}")
    return U


def shifted_tridiag_solve(s, tau, lo, diag, up, r):
    """Solve (s I + tau K) x = r for complex s and r (Thomas, complex128)."""
    r = np.ascontiguousarray(r, dtype=np.complex128)
    n = r.shape[0]
    lo, diag, up = _c(lo), _c(diag), _c(up)
    rr = r.view(np.float64)
    x = np.empty(n, dtype=np.complex128)
    xv = x.view(np.float64)
    rc = lib().or_shifted_tridiag_solve(n, float(np.real(s)), float(np.imag(s)), float(tau),
                                        _p(lo), _p(diag), _p(up), _p(rr), _p(xv))
    if rc != 0:
        raise RuntimeError(f"or_shifted_tridiag_solve failed with code {rc}")
    return x
