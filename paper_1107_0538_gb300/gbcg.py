"""ctypes binding of libgbcg.so, the C ABI declared in include/gbcg.h.

The functions below carry the C names and do argument marshalling only: every
step of a solve runs in the library's CUDA kernels.  ``Solver`` is a small
convenience wrapper that takes a CSR matrix with numpy arrays and torch CUDA
tensors (PyTorch provides device memory and the stream; nothing else).

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1107_0538_gb300.build``); loading fails loudly otherwise.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GBCG_LIBRARY=check loads the bounds-check build (libgbcg_check.so) instead.
LIB_PATH = os.path.join(_HERE, "libgbcg_check.so" if os.environ.get("GBCG_LIBRARY") == "check" else "libgbcg.so")

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA = 0, 1, 2, 3
CG_ENOCONV, CG_EBREAKDOWN, CG_ENAN, CG_ETIMEOUT = 4, 5, 6, 7
CG_MEM_HOST, CG_MEM_DEVICE = 0, 1
CG_PRECOND_NONE, CG_PRECOND_JACOBI, CG_PRECOND_LEARNED = 0, 1, 2
CG_VALUES_FP64, CG_VALUES_FP32, CG_VALUES_BF16 = 0, 1, 2

# Every entry point of include/gbcg.h (checked against the header by the tests).
EXPORTS = ("cg_version", "cg_opts_default", "cg_create", "cg_solve", "cg_solve_host",
           "cg_spmv", "cg_spmv_inner", "cg_get_plan", "cg_destroy", "cg_strerror", "cg_bounds_faults", "cg_fp64_peak",
           "cg_solve_noalloc",
           "cg_batch_create", "cg_batch_enqueue", "cg_batch_results", "cg_batch_solve",
           "cg_batch_tune", "cg_batch_set_tuning", "cg_batch_destroy", "cg_net_create", "cg_net_get_params",
           "cg_net_set_params", "cg_net_destroy", "cg_set_learned", "cg_precond_apply", "cg_learn_pairs",
           "cg_learn_grad", "cg_learn_train")
CG_NOALLOC_MAX_N = 262144
CG_LEARN_PARAMS = 7792


class GbcgError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {cg_strerror(code)} (status {code})" if what else cg_strerror(code))


class cg_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("mem", ctypes.c_int32)]


class cg_opts(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int32), ("true_residual", ctypes.c_int32),
                ("wait_limit_s", ctypes.c_double), ("grid_ctas", ctypes.c_int32),
                ("debug_phantom_arrivals", ctypes.c_int32), ("vectors_in_memory", ctypes.c_int32),
                ("inner_values", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32)]


class cg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("relres", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("launches", ctypes.c_int32), ("outer", ctypes.c_int32),
                ("reverted_at", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class cg_plan(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("ctas", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("tiles", ctypes.c_int32), ("tile_nnz", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("l2_evict_first", ctypes.c_int32),
                ("reg_rows", ctypes.c_int32), ("window_tiles", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("slice_solve", ctypes.c_int32),
                ("inner_solve", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class cg_batch_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("relres", ctypes.c_double)]


class cg_batch_tuning(ctypes.Structure):
    _fields_ = [("inner_tol", ctypes.c_double), ("gather_tiles", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("lanes_per_row", ctypes.c_int32), ("static_split", ctypes.c_int32)]


class cg_learn_set(ctypes.Structure):
    _fields_ = [("ninst", ctypes.c_int32), ("inst", ctypes.c_void_p), ("npairs", ctypes.c_int64),
                ("pair_inst", ctypes.c_void_p), ("r", ctypes.c_void_p), ("e", ctypes.c_void_p)]


_LIB = None
_LOCK = threading.Lock()


def lib() -> ctypes.CDLL:
    """Loads libgbcg.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(the solver has no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
            L.cg_version.argtypes = []
            L.cg_version.restype = ctypes.c_int
            L.cg_opts_default.argtypes = [ctypes.POINTER(cg_opts)]
            L.cg_opts_default.restype = ctypes.c_int
            L.cg_create.argtypes = [ctypes.POINTER(cg_csr), ctypes.POINTER(cg_opts), vp,
                                    ctypes.POINTER(vp)]
            L.cg_create.restype = ctypes.c_int
            for name in ("cg_solve", "cg_solve_host"):
                f = getattr(L, name)
                f.argtypes = [vp, vp, vp, dbl, i32, ctypes.POINTER(cg_info)]
                f.restype = ctypes.c_int
            L.cg_spmv.argtypes = [vp, vp, vp]
            L.cg_spmv.restype = ctypes.c_int
            L.cg_spmv_inner.argtypes = [vp, vp, vp]
            L.cg_spmv_inner.restype = ctypes.c_int
            L.cg_get_plan.argtypes = [vp, ctypes.POINTER(cg_plan)]
            L.cg_get_plan.restype = ctypes.c_int
            L.cg_destroy.argtypes = [vp]
            L.cg_destroy.restype = None
            L.cg_strerror.argtypes = [ctypes.c_int]
            L.cg_strerror.restype = ctypes.c_char_p
            L.cg_bounds_faults.argtypes = [ctypes.POINTER(ctypes.c_int64)]
            L.cg_bounds_faults.restype = ctypes.c_int
            L.cg_fp64_peak.argtypes = [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
            L.cg_fp64_peak.restype = ctypes.c_int
            L.cg_solve_noalloc.argtypes = [ctypes.POINTER(cg_csr), vp, vp, dbl, i32, vp,
                                           ctypes.POINTER(cg_info)]
            L.cg_solve_noalloc.restype = ctypes.c_int
            L.cg_batch_create.argtypes = [ctypes.POINTER(cg_csr), i32, ctypes.POINTER(cg_opts), vp,
                                          ctypes.POINTER(vp)]
            L.cg_batch_create.restype = ctypes.c_int
            L.cg_batch_enqueue.argtypes = [vp, vp, vp, i32, dbl, i32]
            L.cg_batch_enqueue.restype = ctypes.c_int
            L.cg_batch_results.argtypes = [vp, ctypes.POINTER(cg_batch_result)]
            L.cg_batch_results.restype = ctypes.c_int
            L.cg_batch_solve.argtypes = [vp, vp, vp, i32, dbl, i32, ctypes.POINTER(cg_batch_result),
                                         ctypes.POINTER(dbl)]
            L.cg_batch_solve.restype = ctypes.c_int
            L.cg_batch_tune.argtypes = [vp, vp, vp, i32, dbl, ctypes.POINTER(cg_batch_tuning)]
            L.cg_batch_tune.restype = ctypes.c_int
            L.cg_batch_set_tuning.argtypes = [vp, ctypes.POINTER(cg_batch_tuning)]
            L.cg_batch_set_tuning.restype = ctypes.c_int
            L.cg_batch_destroy.argtypes = [vp]
            L.cg_batch_destroy.restype = None
            fp = ctypes.POINTER(ctypes.c_float)
            L.cg_net_create.argtypes = [vp, ctypes.POINTER(vp)]
            L.cg_net_create.restype = ctypes.c_int
            L.cg_net_get_params.argtypes = [vp, vp]
            L.cg_net_get_params.restype = ctypes.c_int
            L.cg_net_set_params.argtypes = [vp, vp]
            L.cg_net_set_params.restype = ctypes.c_int
            L.cg_net_destroy.argtypes = [vp]
            L.cg_net_destroy.restype = None
            L.cg_set_learned.argtypes = [vp, vp, i32, i32, i32, vp, i32, dbl]
            L.cg_set_learned.restype = ctypes.c_int
            L.cg_precond_apply.argtypes = [vp, vp, vp]
            L.cg_precond_apply.restype = ctypes.c_int
            L.cg_learn_pairs.argtypes = [vp, vp, vp, i32, i32, vp, vp]
            L.cg_learn_pairs.restype = ctypes.c_int
            L.cg_learn_grad.argtypes = [vp, ctypes.POINTER(cg_learn_set), vp, i32, ctypes.POINTER(dbl), vp]
            L.cg_learn_grad.restype = ctypes.c_int
            L.cg_learn_train.argtypes = [vp, ctypes.POINTER(cg_learn_set), vp, i32, i32, ctypes.c_float, vp]
            L.cg_learn_train.restype = ctypes.c_int
            del fp
            _LIB = L
    return _LIB


# ---------------------------------------------------------------- C names

def cg_version() -> int:
    return lib().cg_version()


def cg_opts_default() -> cg_opts:
    o = cg_opts()
    rc = lib().cg_opts_default(ctypes.byref(o))
    if rc:
        raise GbcgError(rc, "cg_opts_default")
    return o


def cg_create(A: cg_csr, opts: cg_opts | None, stream: int | None) -> tuple[int, int | None]:
    """Returns (status, handle); handle is None on failure."""
    h = ctypes.c_void_p()
    rc = lib().cg_create(ctypes.byref(A), ctypes.byref(opts) if opts is not None else None,
                         ctypes.c_void_p(stream or 0), ctypes.byref(h))
    return rc, (h.value if rc == CG_OK else None)


def cg_solve(h: int, b_ptr: int, x_ptr: int, tol: float, maxit: int) -> tuple[int, cg_info]:
    info = cg_info()
    rc = lib().cg_solve(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                        float(tol), int(maxit), ctypes.byref(info))
    return rc, info


def cg_solve_host(h: int, b_ptr: int, x_ptr: int, tol: float, maxit: int) -> tuple[int, cg_info]:
    info = cg_info()
    rc = lib().cg_solve_host(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                             float(tol), int(maxit), ctypes.byref(info))
    return rc, info


def cg_spmv(h: int, x_ptr: int, y_ptr: int) -> int:
    return lib().cg_spmv(ctypes.c_void_p(h), ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr))


def cg_spmv_inner(h: int, x_ptr: int, y_ptr: int) -> int:
    return lib().cg_spmv_inner(ctypes.c_void_p(h), ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr))


def cg_get_plan(h: int) -> cg_plan:
    p = cg_plan()
    rc = lib().cg_get_plan(ctypes.c_void_p(h), ctypes.byref(p))
    if rc:
        raise GbcgError(rc, "cg_get_plan")
    return p


def cg_destroy(h: int | None) -> None:
    lib().cg_destroy(ctypes.c_void_p(h or 0))


def cg_strerror(code: int) -> str:
    return lib().cg_strerror(int(code)).decode()


def cg_bounds_faults() -> int:
    """Index faults counted by the bounds-check build (-1: a normal build)."""
    c = ctypes.c_int64(0)
    rc = lib().cg_bounds_faults(ctypes.byref(c))
    if rc != CG_OK:
        raise GbcgError(rc, "cg_bounds_faults")
    return int(c.value)


def cg_fp64_peak(stream: int | None, iters: int) -> tuple[int, float, float]:
    """(status, flops, ms) of the FP64 FMA throughput probe on the current device."""
    flops = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    rc = lib().cg_fp64_peak(ctypes.c_void_p(stream or 0), int(iters), ctypes.byref(flops), ctypes.byref(ms))
    return rc, flops.value, ms.value


def cg_solve_noalloc(A: cg_csr, b_ptr: int, x_ptr: int, tol: float, maxit: int,
                     stream: int | None) -> tuple[int, cg_info]:
    """The allocation-free solve (device CSR and vectors; see include/gbcg.h)."""
    info = cg_info()
    rc = lib().cg_solve_noalloc(ctypes.byref(A), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                                float(tol), int(maxit), ctypes.c_void_p(stream or 0), ctypes.byref(info))
    return rc, info


# ------------------------------------------------------------ convenience

def host_csr(A) -> tuple[cg_csr, tuple]:
    """cg_csr over host numpy copies of A (returned too, to keep them alive)."""
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    vals = np.ascontiguousarray(A.vals, dtype=np.float64)
    c = cg_csr(int(A.n), int(rowptr[-1]) if A.n > 0 else int(colidx.size),
               rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data, CG_MEM_HOST)
    return c, (rowptr, colidx, vals)


class Solver:
    """One CSR matrix on the current CUDA device, solved through the C ABI.

    ``b`` and ``x`` of ``solve`` are float64 CUDA tensors (torch); ``solve_host``
    takes numpy arrays.  The stream is the torch stream current at creation.
    """

    def __init__(self, A, precond: int = CG_PRECOND_NONE, true_residual: bool = True,
                 wait_limit_s: float = 5.0, grid_ctas: int = 0, debug_phantom_arrivals: int = 0,
                 vectors_in_memory: bool = False, inner_values: int = CG_VALUES_FP64,
                 inner_tol: float = 0.0, max_outer: int = 50, max_inner: int = 0, stream=None):
        import torch
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o = cg_opts_default()
        o.precond = precond
        o.true_residual = 1 if true_residual else 0
        o.wait_limit_s = wait_limit_s
        o.grid_ctas = grid_ctas
        o.debug_phantom_arrivals = debug_phantom_arrivals
        o.vectors_in_memory = 1 if vectors_in_memory else 0
        o.inner_values = inner_values
        o.inner_tol = inner_tol
        o.max_outer = max_outer
        o.max_inner = max_inner
        csr, self._keep = host_csr(A)
        rc, self.h = cg_create(csr, o, self.stream.cuda_stream)
        if rc != CG_OK:
            raise GbcgError(rc, "cg_create")
        self.n = int(A.n)

    def solve(self, b, x, tol: float, maxit: int = 0, check: bool = False) -> cg_info:
        t = self._torch
        assert b.dtype == t.float64 and x.dtype == t.float64 and b.is_cuda and x.is_cuda
        assert b.is_contiguous() and x.is_contiguous() and b.numel() == self.n == x.numel()
        rc, info = cg_solve(self.h, b.data_ptr(), x.data_ptr(), tol, maxit)
        if check and rc not in (CG_OK,):
            raise GbcgError(rc, "cg_solve")
        return info

    def solve_host(self, b: np.ndarray, x: np.ndarray, tol: float, maxit: int = 0) -> cg_info:
        assert b.dtype == np.float64 and x.dtype == np.float64
        assert b.flags.c_contiguous and x.flags.c_contiguous and b.size == self.n == x.size
        rc, info = cg_solve_host(self.h, b.ctypes.data, x.ctypes.data, tol, maxit)
        return info

    def spmv(self, x, y) -> None:
        rc = cg_spmv(self.h, x.data_ptr(), y.data_ptr())
        if rc != CG_OK:
            raise GbcgError(rc, "cg_spmv")

    def spmv_inner(self, x, y) -> None:
        """y = A_lo x (float32 CUDA tensors) on a mixed-precision handle."""
        rc = cg_spmv_inner(self.h, x.data_ptr(), y.data_ptr())
        if rc != CG_OK:
            raise GbcgError(rc, "cg_spmv_inner")

    def plan(self) -> dict:
        return cg_get_plan(self.h).as_dict()

    def close(self) -> None:
        if getattr(self, "h", None):
            cg_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches

def cg_batch_create(systems, opts: cg_opts | None, stream: int | None) -> tuple[int, int | None]:
    """systems: a ctypes array of cg_csr.  Returns (status, handle)."""
    h = ctypes.c_void_p()
    rc = lib().cg_batch_create(systems, len(systems), ctypes.byref(opts) if opts is not None else None,
                               ctypes.c_void_p(stream or 0), ctypes.byref(h))
    return rc, (h.value if rc == CG_OK else None)


def cg_batch_enqueue(h: int, b_ptr: int, x_ptr: int, nrhs: int, tol: float, maxit: int) -> int:
    return lib().cg_batch_enqueue(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                                  int(nrhs), float(tol), int(maxit))


def cg_batch_results(h: int, nsys: int, nrhs: int) -> tuple[int, list]:
    res = (cg_batch_result * (nsys * nrhs))()
    rc = lib().cg_batch_results(ctypes.c_void_p(h), res)
    return rc, list(res)


def cg_batch_solve(h: int, b_ptr: int, x_ptr: int, nsys: int, nrhs: int, tol: float,
                   maxit: int) -> tuple[int, list, float]:
    res = (cg_batch_result * (nsys * nrhs))()
    ms = ctypes.c_double(0.0)
    rc = lib().cg_batch_solve(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                              int(nrhs), float(tol), int(maxit), res, ctypes.byref(ms))
    return rc, list(res), ms.value


def cg_batch_tune(h: int, b_ptr: int, x_ptr: int, nrhs: int, tol: float) -> tuple[int, cg_batch_tuning]:
    t = cg_batch_tuning()
    rc = lib().cg_batch_tune(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr),
                             int(nrhs), float(tol), ctypes.byref(t))
    return rc, t


def cg_batch_set_tuning(h: int, choice: cg_batch_tuning) -> int:
    return lib().cg_batch_set_tuning(ctypes.c_void_p(h), ctypes.byref(choice))


def cg_batch_destroy(h: int | None) -> None:
    lib().cg_batch_destroy(ctypes.c_void_p(h or 0))


class BatchSolver:
    """Independent systems (CSR objects with numpy arrays) solved together on
    the current CUDA device; right-hand sides and solutions are float64 torch
    tensors of shape (nrhs, N), N the total row count (systems concatenated)."""

    def __init__(self, systems, inner_values: int = CG_VALUES_FP32, precond: int = CG_PRECOND_NONE,
                 inner_tol: float = 0.0, max_outer: int = 50, max_inner: int = 0, grid_ctas: int = 0,
                 stream=None):
        import torch
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o = cg_opts_default()
        o.inner_values = inner_values
        o.precond = precond
        o.inner_tol = inner_tol
        o.max_outer = max_outer
        o.max_inner = max_inner
        o.grid_ctas = grid_ctas
        arr = (cg_csr * len(systems))()
        self._keep = []
        for i, A in enumerate(systems):
            c, keep = host_csr(A)
            arr[i] = c
            self._keep.append(keep)
        rc, self.h = cg_batch_create(arr, o, self.stream.cuda_stream)
        if rc != CG_OK:
            raise GbcgError(rc, "cg_batch_create")
        self.nsys = len(systems)
        self.sizes = [int(A.n) for A in systems]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])

    def solve(self, B, X, tol: float, maxit: int = 0):
        assert B.shape == X.shape and B.shape[1] == self.n and B.is_contiguous() and X.is_contiguous()
        rc, res, ms = cg_batch_solve(self.h, B.data_ptr(), X.data_ptr(), self.nsys, B.shape[0], tol, maxit)
        return rc, res, ms

    def enqueue(self, B, X, tol: float, maxit: int = 0) -> int:
        return cg_batch_enqueue(self.h, B.data_ptr(), X.data_ptr(), B.shape[0], tol, maxit)

    def results(self, nrhs: int):
        return cg_batch_results(self.h, self.nsys, nrhs)

    def tune(self, B, X, tol: float):
        return cg_batch_tune(self.h, B.data_ptr(), X.data_ptr(), B.shape[0], tol)

    def set_tuning(self, inner_tol: float, gather_tiles: int, lanes_per_row: int, static_split: int = 0) -> None:
        c = cg_batch_tuning(inner_tol=inner_tol, gather_tiles=gather_tiles, lanes_per_row=lanes_per_row,
                            static_split=static_split)
        rc = cg_batch_set_tuning(self.h, c)
        if rc != CG_OK:
            raise GbcgError(rc, "cg_batch_set_tuning")

    def close(self) -> None:
        if getattr(self, "h", None):
            cg_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------ learned preconditioner

def cg_net_create(params: np.ndarray) -> tuple[int, int | None]:
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == CG_LEARN_PARAMS
    h = ctypes.c_void_p()
    rc = lib().cg_net_create(ctypes.c_void_p(p.ctypes.data), ctypes.byref(h))
    return rc, (h.value if rc == CG_OK else None)


def cg_net_get_params(net: int) -> tuple[int, np.ndarray]:
    out = np.zeros(CG_LEARN_PARAMS, dtype=np.float32)
    rc = lib().cg_net_get_params(ctypes.c_void_p(net), ctypes.c_void_p(out.ctypes.data))
    return rc, out


def cg_net_set_params(net: int, params: np.ndarray) -> int:
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == CG_LEARN_PARAMS
    return lib().cg_net_set_params(ctypes.c_void_p(net), ctypes.c_void_p(p.ctypes.data))


def cg_net_destroy(net: int | None) -> None:
    lib().cg_net_destroy(ctypes.c_void_p(net or 0))


def cg_set_learned(h: int, net: int, ex: int, ey: int, ez: int, lognu: np.ndarray, stall_window: int = 0,
                   stall_factor: float = 0.0) -> int:
    ln = np.ascontiguousarray(lognu, dtype=np.float32)
    return lib().cg_set_learned(ctypes.c_void_p(h), ctypes.c_void_p(net), int(ex), int(ey), int(ez),
                                ctypes.c_void_p(ln.ctypes.data), int(stall_window), float(stall_factor))


def cg_precond_apply(h: int, r_ptr: int, z_ptr: int) -> int:
    return lib().cg_precond_apply(ctypes.c_void_p(h), ctypes.c_void_p(r_ptr), ctypes.c_void_p(z_ptr))


def cg_learn_pairs(h: int, b_ptr: int, xstar_ptr: int, segment: int, count: int, r_ptr: int, e_ptr: int) -> int:
    return lib().cg_learn_pairs(ctypes.c_void_p(h), ctypes.c_void_p(b_ptr), ctypes.c_void_p(xstar_ptr),
                                int(segment), int(count), ctypes.c_void_p(r_ptr), ctypes.c_void_p(e_ptr))


def cg_learn_grad(net: int, lset: cg_learn_set, pairs: np.ndarray) -> tuple[int, float, np.ndarray]:
    pr = np.ascontiguousarray(pairs, dtype=np.int64)
    loss = ctypes.c_double(0.0)
    grad = np.zeros(CG_LEARN_PARAMS, dtype=np.float32)
    rc = lib().cg_learn_grad(ctypes.c_void_p(net), ctypes.byref(lset), ctypes.c_void_p(pr.ctypes.data),
                             int(pr.size), ctypes.byref(loss), ctypes.c_void_p(grad.ctypes.data))
    return rc, loss.value, grad


def cg_learn_train(net: int, lset: cg_learn_set, order: np.ndarray, steps: int, batch: int,
                   lr: float) -> tuple[int, np.ndarray]:
    od = np.ascontiguousarray(order, dtype=np.int64)
    assert od.size >= steps * batch
    losses = np.zeros(steps, dtype=np.float64)
    rc = lib().cg_learn_train(ctypes.c_void_p(net), ctypes.byref(lset), ctypes.c_void_p(od.ctypes.data),
                              int(steps), int(batch), ctypes.c_float(lr), ctypes.c_void_p(losses.ctypes.data))
    return rc, losses


class Net:
    """The learned preconditioner's parameters on the current CUDA device."""

    def __init__(self, params: np.ndarray):
        rc, self.h = cg_net_create(params)
        if rc != CG_OK:
            raise GbcgError(rc, "cg_net_create")

    def params(self) -> np.ndarray:
        rc, p = cg_net_get_params(self.h)
        if rc != CG_OK:
            raise GbcgError(rc, "cg_net_get_params")
        return p

    def set_params(self, params: np.ndarray) -> None:
        rc = cg_net_set_params(self.h, params)
        if rc != CG_OK:
            raise GbcgError(rc, "cg_net_set_params")

    def grad(self, lset: "LearnSet", pairs) -> tuple[float, np.ndarray]:
        rc, loss, g = cg_learn_grad(self.h, lset.c, np.asarray(pairs))
        if rc != CG_OK:
            raise GbcgError(rc, "cg_learn_grad")
        return loss, g

    def train(self, lset: "LearnSet", order, steps: int, batch: int, lr: float) -> np.ndarray:
        rc, losses = cg_learn_train(self.h, lset.c, np.asarray(order), steps, batch, lr)
        if rc != CG_OK:
            raise GbcgError(rc, "cg_learn_train")
        return losses

    def close(self) -> None:
        if getattr(self, "h", None):
            cg_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LearnSet:
    """Training pairs (float32 CUDA tensors R, E of shape (npairs, n)) over
    learned Solvers that share one grid; pair_inst gives each pair's solver."""

    def __init__(self, solvers, pair_inst, R, E):
        self._inst = (ctypes.c_void_p * len(solvers))(*[s.h for s in solvers])
        self._pi = np.ascontiguousarray(pair_inst, dtype=np.int32)
        assert R.shape == E.shape and R.shape[0] == self._pi.size and R.is_contiguous() and E.is_contiguous()
        self._keep = (solvers, R, E)
        self.c = cg_learn_set(len(solvers), ctypes.cast(self._inst, ctypes.c_void_p), int(self._pi.size),
                              self._pi.ctypes.data, R.data_ptr(), E.data_ptr())


def _solver_set_learned(self, net: Net, grid, lognu: np.ndarray, stall_window: int = 0,
                        stall_factor: float = 0.0) -> None:
    """Attaches the learned preconditioner (grid: object with ex, ey, ez)."""
    rc = cg_set_learned(self.h, net.h, grid.ex, grid.ey, grid.ez, lognu, stall_window, stall_factor)
    if rc != CG_OK:
        raise GbcgError(rc, "cg_set_learned")
    self._net = net


def _solver_precond_apply(self, r, z) -> None:
    rc = cg_precond_apply(self.h, r.data_ptr(), z.data_ptr())
    if rc != CG_OK:
        raise GbcgError(rc, "cg_precond_apply")


def _solver_learn_pairs(self, b, xstar, segment: int, count: int, R, E) -> None:
    rc = cg_learn_pairs(self.h, b.data_ptr(), xstar.data_ptr(), segment, count, R.data_ptr(), E.data_ptr())
    if rc != CG_OK:
        raise GbcgError(rc, "cg_learn_pairs")


Solver.set_learned = _solver_set_learned
Solver.precond_apply = _solver_precond_apply
Solver.learn_pairs = _solver_learn_pairs
