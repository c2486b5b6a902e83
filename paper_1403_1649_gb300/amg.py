"""Thin ctypes binding of the C ABI in ``include/amg.h`` (same names).

Argument marshalling only: every step of setup and solve runs in the CUDA
library ``_build/libamg_gb300.so``.  There is no CPU fallback; if the library
is missing this module raises at import of the library.

Arrays may be numpy arrays (host memory; the library copies them in and out)
or CUDA torch tensors (device memory, used in place on the current stream).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libamg_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "amg.h")

AMG_OK = 0
AMG_ERR_BAD_INPUT = -1
AMG_ERR_CUDA = -2
AMG_ERR_NOT_CONVERGED = -3
AMG_ERR_BREAKDOWN = -4
AMG_ERR_NAN = -5
AMG_ERR_SETUP = -6
AMG_ERR_UNSUPPORTED = -7
AMG_PREC_F64, AMG_PREC_F32, AMG_PREC_BF16 = 0, 1, 2


class amg_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class amg_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("seed", C.c_uint64), ("coarse_max", C.c_int32),
                ("max_levels", C.c_int32), ("kcycle_levels", C.c_int32), ("kcycle_t", C.c_double),
                ("omega_mode", C.c_int32), ("omega", C.c_double), ("precision", C.c_int32),
                ("outer", C.c_int32), ("restart", C.c_int32), ("max_iter", C.c_int32),
                ("use_graph", C.c_int32), ("smoother", C.c_int32), ("tail", C.c_int32), ("pdl", C.c_int32),
                ("autotune", C.c_int32), ("symmetric", C.c_int32), ("mis_k", C.c_int32)]


class amg_level_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("n_coarse", C.c_int32), ("mis_rounds", C.c_int32),
                ("omega", C.c_double), ("spmv_blocks", C.c_int32), ("seg_tile", C.c_int32)]


class amg_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("final_relres", C.c_double),
                ("solve_ms", C.c_double), ("setup_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("setup_launches", C.c_int64)]


class AMGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"AMG error {code}: {msg}")
        self.code = code


_lib = None


def lib() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not found: build it with __graft_entry__.build() "
                              "(the GPU path has no fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.amg_default_params.argtypes = [C.POINTER(amg_params)]
        L.amg_default_params.restype = None
        L.amg_setup.argtypes = [C.POINTER(amg_csr), C.POINTER(amg_params), vp, C.POINTER(vp)]
        L.amg_solve.argtypes = [vp, vp, vp, dbl, C.POINTER(i32), vp, vp]
        L.amg_precond.argtypes = [vp, vp, vp, vp]
        L.amg_resetup_values.argtypes = [vp, vp, vp]
        L.amg_spmv.argtypes = [vp, i32, vp, vp, vp]
        L.amg_set_poly.argtypes = [vp, i32, vp, vp]
        L.amg_hierarchy_info.argtypes = [vp, vp, i32, C.POINTER(i32)]
        L.amg_export_level.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.amg_last_solve_info.argtypes = [vp, C.POINTER(amg_solve_info)]
        L.amg_cycle_trace.argtypes = [vp, vp, vp, vp, i32, vp]
        L.amg_free.argtypes = [vp]
        L.amg_free.restype = None
        L.amg_last_error.argtypes = []
        L.amg_last_error.restype = C.c_char_p
        u64 = C.c_uint64
        L.amg_features.argtypes = [vp, i32, vp, vp]
        L.amg_mlp_forward.argtypes = [i32, vp, vp, vp, vp]
        L.amg_mlp_backward.argtypes = [i32, vp, vp, vp, vp, vp]
        L.amg_mlp_backward_noalloc.argtypes = [i32, vp, vp, vp, vp, vp]
        L.amg_mlp_backward_noalloc.restype = C.c_int
        L.amg_twogrid_loss.argtypes = [vp, vp, i32, u64, C.POINTER(dbl), vp, vp]
        L.amg_train_smoother.argtypes = [vp, i32, i32, dbl, i32, u64, vp, vp, vp]
        L.amg_apply_learned_smoother.argtypes = [vp, vp, vp]
        L.amg_setup_batch.argtypes = [i32, vp, C.POINTER(amg_params), vp, C.POINTER(vp)]
        L.amg_solve_batch.argtypes = [vp, vp, vp, dbl, vp, vp, vp]
        L.amg_setup_batch.restype = C.c_int
        L.amg_validate_hierarchy.argtypes = [vp]
        L.amg_validate_hierarchy.restype = C.c_int
        L.amg_solve_batch.restype = C.c_int
        for name in ("amg_setup", "amg_solve", "amg_precond", "amg_resetup_values", "amg_spmv", "amg_set_poly", "amg_hierarchy_info",
                     "amg_export_level", "amg_last_solve_info", "amg_features", "amg_mlp_forward",
                     "amg_mlp_backward", "amg_twogrid_loss", "amg_train_smoother", "amg_apply_learned_smoother"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/amg.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(amg_[a-z_0-9]+)\s*\(", txt)))


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _stream(*arrays):
    for a in arrays:
        if a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False):
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def amg_last_error() -> str:
    return lib().amg_last_error().decode()


def _check(rc: int, ok=(AMG_OK,)) -> int:
    if rc not in ok:
        raise AMGError(rc, amg_last_error())
    return rc


def amg_default_params(**overrides) -> amg_params:
    p = amg_params()
    lib().amg_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def amg_setup(rowptr, col, val, params: amg_params | None = None, stream=None) -> C.c_void_p:
    """Build the hierarchy (Alg. 1) of the CSR matrix; returns an opaque handle."""
    n = len(rowptr) - 1
    nnz = len(col)
    if isinstance(rowptr, np.ndarray):
        rowptr = np.ascontiguousarray(rowptr, np.int32)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float64)
    csr = amg_csr(n, nnz, _ptr(rowptr), _ptr(col), _ptr(val))
    h = C.c_void_p()
    p = params if params is not None else amg_default_params()
    _check(lib().amg_setup(C.byref(csr), C.byref(p), stream if stream is not None else _stream(rowptr),
                           C.byref(h)))
    return h


def amg_setup_batch(systems, params: amg_params | None = None, stream=None) -> C.c_void_p:
    """Block-diagonal hierarchy of independent systems (list of CSR objects or
    (rowptr, col, val) triples, numpy or CUDA tensors)."""
    arr = (amg_csr * len(systems))()
    keep = []
    for q, A in enumerate(systems):
        rp, ci, va = (A.rowptr, A.col, A.val) if hasattr(A, "rowptr") else A
        if isinstance(rp, np.ndarray):
            rp = np.ascontiguousarray(rp, np.int32)
            ci = np.ascontiguousarray(ci, np.int32)
            va = np.ascontiguousarray(va, np.float64)
        keep.append((rp, ci, va))
        arr[q] = amg_csr(len(rp) - 1, len(ci), _ptr(rp), _ptr(ci), _ptr(va))
    h = C.c_void_p()
    p = params if params is not None else amg_default_params()
    _check(lib().amg_setup_batch(len(systems), arr, C.byref(p), stream, C.byref(h)))
    return h


def amg_solve_batch(h, b, x, tol: float, nsys: int, stream=None, allow=(AMG_OK,)):
    """Solve every system of a batch; b, x concatenated.  Returns (status, iters, relres)."""
    if isinstance(b, np.ndarray):
        b = np.ascontiguousarray(b, np.float64)
    it = np.zeros(nsys, np.int32)
    rel = np.zeros(nsys)
    rc = lib().amg_solve_batch(h, _ptr(b), _ptr(x), tol, it.ctypes.data, rel.ctypes.data,
                               stream if stream is not None else _stream(b, x))
    _check(rc, allow)
    return rc, it, rel


def amg_solve(h, b, x, tol: float, max_iter: int | None = None, stream=None, allow=(AMG_OK,)):
    """Solve A x = b (x holds x0 and receives the solution).  Returns (status, iters, hist)."""
    if isinstance(b, np.ndarray):
        b = np.ascontiguousarray(b, np.float64)
        assert x.dtype == np.float64 and x.flags.c_contiguous
    it = C.c_int32()
    cap = (max_iter or 100000) + 1
    hist = np.zeros(cap)
    rc = lib().amg_solve(h, _ptr(b), _ptr(x), tol, C.byref(it), hist.ctypes.data,
                         stream if stream is not None else _stream(b, x))
    _check(rc, allow)
    return rc, it.value, hist[:it.value + 1].copy()


def amg_resetup_values(h, val, stream=None) -> None:
    """Values-only re-setup with new values of A_0 (same pattern, CSR order)."""
    if isinstance(val, np.ndarray):
        val = np.ascontiguousarray(val, np.float64)
    _check(lib().amg_resetup_values(h, _ptr(val), stream if stream is not None else _stream(val)))


def amg_precond(h, b, x, stream=None) -> None:
    _check(lib().amg_precond(h, _ptr(b), _ptr(x), stream if stream is not None else _stream(b, x)))


def amg_spmv(h, level: int, x, y, stream=None) -> None:
    _check(lib().amg_spmv(h, level, _ptr(x), _ptr(y), stream if stream is not None else _stream(x, y)))


def amg_set_poly(h, level: int, coef, stream=None) -> None:
    if isinstance(coef, np.ndarray):
        coef = np.ascontiguousarray(coef, np.float64)
    _check(lib().amg_set_poly(h, level, _ptr(coef), stream if stream is not None else _stream(coef)))


def amg_hierarchy_info(h) -> list[dict]:
    nl = C.c_int32()
    _check(lib().amg_hierarchy_info(h, None, 0, C.byref(nl)))
    arr = (amg_level_info * nl.value)()
    _check(lib().amg_hierarchy_info(h, arr, nl.value, C.byref(nl)))
    return [{"n": a.n, "nnz": a.nnz, "n_coarse": a.n_coarse, "mis_rounds": a.mis_rounds, "omega": a.omega,
             "spmv_blocks": a.spmv_blocks, "seg_tile": a.seg_tile} for a in arr]


def amg_export_level(h, level: int) -> dict:
    info = amg_hierarchy_info(h)[level]
    n, nnz = info["n"], info["nnz"]
    last = info["n_coarse"] == 0
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1))
    agg = np.zeros(n, np.int32)
    P = np.zeros(n)
    B = np.zeros(n)
    _check(lib().amg_export_level(h, level, rp.ctypes.data, ci.ctypes.data, val.ctypes.data, agg.ctypes.data,
                                  P.ctypes.data, B.ctypes.data))
    return {"n": n, "nnz": nnz, "rowptr": rp, "col": ci[:nnz], "val": val[:nnz],
            "agg": None if last else agg, "P": None if last else P, "B": B, "omega": info["omega"],
            "mis_rounds": info["mis_rounds"]}


def amg_last_solve_info(h) -> dict:
    s = amg_solve_info()
    _check(lib().amg_last_solve_info(h, C.byref(s)))
    return {k: getattr(s, k) for k, _ in amg_solve_info._fields_}


def amg_cycle_trace(h) -> dict:
    """Per level: cycle visits, Alg. 5 coarse parts run, second inner steps taken (last solve)."""
    nl = C.c_int32()
    _check(lib().amg_hierarchy_info(h, None, 0, C.byref(nl)))
    v, k, s2 = (np.zeros(nl.value, np.int64) for _ in range(3))
    _check(lib().amg_cycle_trace(h, v.ctypes.data, k.ctypes.data, s2.ctypes.data, nl.value, None))
    return {"visits": v, "kcalls": k, "second": s2}


def amg_free(h) -> None:
    if h:
        lib().amg_free(h)


class Hierarchy:
    """Owning wrapper around an amg_hierarchy handle."""

    def __init__(self, A, params: amg_params | None = None, **overrides):
        p = params if params is not None else amg_default_params(**overrides)
        self.params = p
        self.n = A.n
        self.h = amg_setup(A.rowptr, A.col, A.val, p)

    def __del__(self):
        if getattr(self, "h", None):
            amg_free(self.h)
            self.h = None

    def free(self):
        self.__del__()

    @property
    def nlevels(self) -> int:
        return len(amg_hierarchy_info(self.h))

    def info(self):
        return amg_hierarchy_info(self.h)

    def level(self, k: int) -> dict:
        return amg_export_level(self.h, k)

    def solve(self, b, x0=None, tol: float = 1e-8, allow=(AMG_OK,)):
        x = np.zeros(self.n) if x0 is None else (x0.copy() if isinstance(x0, np.ndarray) else x0.clone())
        rc, it, hist = amg_solve(self.h, b, x, tol, self.params.max_iter, allow=allow)
        return x, {"status": rc, "iters": it, "hist": hist, **amg_last_solve_info(self.h)}

    def precond(self, b):
        x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.clone()
        amg_precond(self.h, b, x)
        return x
