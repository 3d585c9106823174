"""CPU FP64 oracle for the conjugate-gradient hot path (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  The
product path (``paper_1107_0538_gb300``) never imports it, and this package
never imports the product path: the two share only the seeded input
generators, which hold none of the solver's arithmetic.

The arithmetic lives in ``cg_oracle.c`` (plain serial C, FP64, no fused
multiply-add, sums left to right).  This module compiles it with gcc on first
use and marshals numpy arrays to it with ctypes.

Parity status of each function (what pins it is in ``tests/test_oracle.py``):
  spmv, cg (plain and Jacobi), round_to_format  -- pinned
  lowprec_values                                -- pinned (row sums, SPD, format)
  cg_ir                                         -- pinned (reduces to CG; exact-solve limit)

``cg_omp`` (``cg_omp.c``, built with OpenMP) is not part of the oracle: it is
the multi-core CPU baseline that ``bench.py`` times on all host cores.  It
sums its dot products per thread, so its rounding differs from ``cg``; its
test checks it against ``cg``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_OMP_SRC = os.path.join(_HERE, "cg_omp.c")
_OMP_SO = os.path.join(_HERE, "libcg_omp.so")
_LOCK = threading.Lock()
_LIB = None
_OMP = None

OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN, ENAN = 0, 1, 2, 4, 5, 6
STATUS_NAMES = {OK: "ok", EINVAL: "einval", ENOMEM: "enomem", ENOCONV: "enoconv",
                EBREAKDOWN: "ebreakdown", ENAN: "enan"}

# (significand bits incl. hidden bit, min normal exponent, max exponent)
FP32_FORMAT = (24, -126, 127)
BF16_FORMAT = (8, -126, 127)


def build(force: bool = False) -> str:
    """Compile cg_oracle.c into liboracle.so next to it (gcc, no FMA contraction),
    and the OpenMP baseline cg_omp.c into libcg_omp.so."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    if force or not os.path.exists(_OMP_SO) or os.path.getmtime(_OMP_SO) < os.path.getmtime(_OMP_SRC):
        tmp = _OMP_SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _OMP_SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OMP_SO)
    return _SO


def _omp():
    global _OMP
    with _LOCK:
        if _OMP is None:
            build()
            lib = ctypes.CDLL(_OMP_SO)
            i32, dbl, vp = ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.cpu_cg_omp.argtypes = [i32, vp, vp, vp, vp, vp, dbl, i32, ctypes.POINTER(i32),
                                       ctypes.POINTER(dbl)]
            lib.cpu_cg_omp.restype = ctypes.c_int
            lib.cpu_omp_threads.argtypes = []
            lib.cpu_omp_threads.restype = ctypes.c_int
            _OMP = lib
    return _OMP


def omp_threads() -> int:
    """Threads the OpenMP baseline runs with (OMP_NUM_THREADS, else all host cores)."""
    return int(_omp().cpu_omp_threads())


def cg_omp(A, b, x0=None, tol: float = 1e-8, maxit: int = 0) -> dict:
    """Plain FP64 CG with OpenMP row and vector loops: the timed multi-core CPU
    baseline, not the parity reference.  Returns dict(x, iters, relres, status)."""
    n, rowptr, colidx, vals = _csr_arrays(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = _omp().cpu_cg_omp(n, _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(b), _ptr(x), float(tol),
                           int(maxit), ctypes.byref(it), ctypes.byref(rel))
    return dict(x=x, iters=int(it.value), relres=float(rel.value), status=int(st))


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.oracle_spmv.argtypes = [i32, vp, vp, vp, vp, vp]
            lib.oracle_spmv.restype = None
            lib.oracle_dot.argtypes = [i32, vp, vp]
            lib.oracle_dot.restype = dbl
            lib.oracle_cg.argtypes = [i32, vp, vp, vp, vp, vp, dbl, i32, i32,
                                      ctypes.POINTER(i32), ctypes.POINTER(dbl), vp, vp, vp]
            lib.oracle_cg.restype = ctypes.c_int
            lib.oracle_round_to_format.argtypes = [dbl, i32, i32, i32]
            lib.oracle_round_to_format.restype = dbl
            lib.oracle_round_array.argtypes = [i64, vp, vp, i32, i32, i32]
            lib.oracle_round_array.restype = None
            lib.oracle_lowprec_values.argtypes = [i32, vp, vp, vp, i32, i32, i32, vp]
            lib.oracle_lowprec_values.restype = None
            lib.oracle_cg_ir.argtypes = [i32, vp, vp, vp, vp, vp, vp, dbl, dbl, i32, i32,
                                         ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(dbl)]
            lib.oracle_cg_ir.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr_arrays(A):
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    vals = np.ascontiguousarray(A.vals, dtype=np.float64)
    return int(A.n), rowptr, colidx, vals


def spmv(A, x) -> np.ndarray:
    """y = A x, one row at a time in storage order (Section IV, "DGEMV(sparse)")."""
    n, rowptr, colidx, vals = _csr_arrays(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    _lib().oracle_spmv(n, _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(x), _ptr(y))
    return y


def dot(a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(_lib().oracle_dot(a.size, _ptr(a), _ptr(b)))


def cg(A, b, x0=None, tol: float = 1e-8, maxit: int = 0, precond: int = 0,
       trace: bool = False) -> dict:
    """Plain (precond=0) or Jacobi-preconditioned (precond=1) CG, Section IV.

    Returns dict(x, iters, relres, status[, xtrace, ptrace, rtrace]).  With
    ``trace`` the iterates x_k, residuals r_k and directions p_k are recorded
    (only for small n: the traces take (maxit + 1) * n doubles each).
    """
    n, rowptr, colidx, vals = _csr_arrays(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    mi = n if maxit <= 0 else int(maxit)
    xt = pt = rt = None
    if trace:
        xt = np.full((mi + 1, n), np.nan)
        pt = np.full((max(mi, 1), n), np.nan)
        rt = np.full((mi + 1, n), np.nan)
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = _lib().oracle_cg(n, _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(b), _ptr(x),
                          float(tol), int(maxit), int(precond), ctypes.byref(it),
                          ctypes.byref(rel), _ptr(xt), _ptr(pt), _ptr(rt))
    out = dict(x=x, iters=int(it.value), relres=float(rel.value), status=int(st))
    if trace:
        k = int(it.value)
        out.update(xtrace=xt[:k + 1], ptrace=pt[:k], rtrace=rt[:k + 1])
    return out


def round_to_format(v, fmt) -> np.ndarray:
    """Round FP64 values to a binary format (RNE, gradual underflow, overflow to inf)."""
    v = np.ascontiguousarray(np.atleast_1d(v), dtype=np.float64)
    out = np.empty_like(v)
    p, emin, emax = fmt
    _lib().oracle_round_array(v.size, _ptr(v), _ptr(out), p, emin, emax)
    return out


def lowprec_values(A, fmt) -> np.ndarray:
    """Inner-solve matrix values: off-diagonals rounded to ``fmt``, diagonal
    row-sum compensated and rounded to FP32 (see oracle_lowprec_values)."""
    n, rowptr, colidx, vals = _csr_arrays(A)
    out = np.empty_like(vals)
    p, emin, emax = fmt
    _lib().oracle_lowprec_values(n, _ptr(rowptr), _ptr(colidx), _ptr(vals), p, emin, emax,
                                 _ptr(out))
    return out


def cg_ir(A, vals_lo, b, x0=None, tol: float = 1e-8, inner_tol: float = 1e-3,
          max_outer: int = 50, max_inner: int = 0) -> dict:
    """FP64 iterative refinement around CG on a rounded copy of the matrix values."""
    n, rowptr, colidx, vals = _csr_arrays(A)
    vals_lo = np.ascontiguousarray(vals_lo, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    outer = ctypes.c_int32(0)
    inner = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = _lib().oracle_cg_ir(n, _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(vals_lo),
                             _ptr(b), _ptr(x), float(tol), float(inner_tol), int(max_outer),
                             int(max_inner), ctypes.byref(outer), ctypes.byref(inner),
                             ctypes.byref(rel))
    return dict(x=x, outer=int(outer.value), inner=int(inner.value),
                relres=float(rel.value), status=int(st))
