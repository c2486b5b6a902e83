"""ctypes front end of the FP64 CPU oracle (``amg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark use this module.  The GPU library never imports it.

``build()`` compiles the C oracle with ``-O2 -ffp-contract=off`` (no fused
multiply-add, so every operation is rounded exactly as written).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "amg_oracle.c")
LIB = os.path.join(HERE, "_build", "libamg_oracle.so")

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


class ORParams(C.Structure):
    _fields_ = [
        ("alpha", C.c_double),
        ("seed", C.c_uint64),
        ("coarse_max", C.c_int32),
        ("max_levels", C.c_int32),
        ("kcycle_levels", C.c_int32),
        ("kcycle_t", C.c_double),
        ("omega_mode", C.c_int32),
        ("omega", C.c_double),
        ("outer", C.c_int32),
        ("restart", C.c_int32),
        ("smoother", C.c_int32),
        ("symmetric", C.c_int32),
        ("mis_k", C.c_int32),
    ]


LIB_OMP = os.path.join(HERE, "_build", "libamg_oracle_omp.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library, and its OpenMP timing build for the
    benchmark's CPU baseline (idempotent)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    stamp = max(os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "amg_oracle.h")))
    for out, extra in ((LIB, []), (LIB_OMP, ["-fopenmp"])):
        if not force and os.path.exists(out) and os.path.getmtime(out) >= stamp:
            continue
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               *extra, "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, out)
    return LIB


_libs = {}


def lib(omp: bool = False):
    """The parity build, or (omp=True) the OpenMP timing build of the CPU baseline."""
    if omp not in _libs:
        build()
        L = C.CDLL(LIB_OMP if omp else LIB)
        L.or_strength.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, _u8p]
        L.or_col_count.argtypes = [C.c_int32, _i32p, _i32p, _u8p, _i32p]
        L.or_sym_graph.argtypes = [C.c_int32, _i32p, _i32p, _u8p, _i32p, C.c_void_p, C.c_int64]
        L.or_sym_graph.restype = C.c_int64
        L.or_mis_hash.argtypes = [C.c_uint64, C.c_int32, C.c_int32]
        L.or_mis_hash.restype = C.c_uint32
        L.or_splitmix64.argtypes = [C.c_uint64]
        L.or_splitmix64.restype = C.c_uint64
        L.or_pmis.argtypes = [C.c_int32, _i32p, _i32p, _i32p, _u32p, _i8p, C.c_int32]
        L.or_pmis.restype = C.c_int32
        L.or_aggregate.argtypes = [C.c_int32, _i32p, _i32p, _i32p, _u32p, _i8p, _i32p, C.c_int32]
        L.or_aggregate.restype = C.c_int32
        L.or_interp.argtypes = [C.c_int32, C.c_int32, _i32p, _f64p, _f64p, _f64p]
        L.or_galerkin.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, _i32p, C.c_void_p, _i32p,
                                  C.c_void_p, C.c_void_p, C.c_int64]
        L.or_galerkin.restype = C.c_int64
        L.or_rho_estimate.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_uint64, C.c_int32, C.c_int32,
                                      C.c_void_p, C.c_int32]
        L.or_hess_rho.argtypes = [C.c_int32, _f64p]
        L.or_hess_rho.restype = C.c_double
        L.or_lu.argtypes = [C.c_int32, _f64p, _i32p]
        L.or_lu.restype = C.c_int32
        L.or_lu_solve.argtypes = [C.c_int32, _f64p, _i32p, _f64p]
        L.or_rho_estimate.restype = C.c_double
        L.or_sym_eig.argtypes = [C.c_int32, _f64p, _f64p]
        L.or_cholesky.argtypes = [C.c_int32, _f64p]
        L.or_cholesky.restype = C.c_int32
        L.or_chol_solve.argtypes = [C.c_int32, _f64p, _f64p]
        L.or_default_params.argtypes = [C.POINTER(ORParams)]
        L.or_setup.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.POINTER(ORParams), C.POINTER(C.c_int32)]
        L.or_setup.restype = C.c_void_p
        L.or_nlevels.argtypes = [C.c_void_p]
        L.or_nlevels.restype = C.c_int32
        L.or_level_info.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double), C.POINTER(C.c_int32)]
        L.or_level_copy.argtypes = [C.c_void_p, C.c_int32] + [C.c_void_p] * 6
        L.or_set_poly.argtypes = [C.c_void_p, C.c_int32, _f64p]
        L.or_set_poly.restype = C.c_int32
        L.or_precond.argtypes = [C.c_void_p, _f64p, _f64p]
        L.or_solve.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_int32, C.POINTER(C.c_int32), _f64p,
                               C.POINTER(C.c_double)]
        L.or_solve.restype = C.c_int32
        L.or_free.argtypes = [C.c_void_p]
        L.or_subsystem.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
        L.or_cycle_trace.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_subsystem.restype = C.c_void_p
        L.or_krylov2_probe.argtypes = [C.c_void_p, C.c_int32, _f64p, _f64p, _f64p, _f64p]
        L.or_krylov2_probe.restype = C.c_int32
        _f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
        _u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
        L.or_features.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, _f32p]
        L.or_mlp_forward.argtypes = [C.c_int32, _u16p, _f32p, _f32p]
        L.or_mlp_backward.argtypes = [C.c_int32, _f64p, _f32p, _f64p, _f64p, C.c_void_p]
        L.or_twogrid_loss.argtypes = [C.c_void_p, _f64p, C.c_int32, C.c_uint64, C.c_void_p]
        L.or_twogrid_loss.restype = C.c_double
        L.or_threads.restype = C.c_int32
        _libs[omp] = L
    return _libs[omp]


def _csr_args(A):
    return (int(A.n), np.ascontiguousarray(A.rowptr, np.int32), np.ascontiguousarray(A.col, np.int32),
            np.ascontiguousarray(A.val, np.float64))


# ---------------------------------------------------------------- setup steps
def strength(A, alpha: float) -> np.ndarray:
    n, rp, ci, v = _csr_args(A)
    Cm = np.zeros(max(A.nnz, 1), np.uint8)
    lib().or_strength(n, rp, ci, v, alpha, Cm)
    return Cm[:A.nnz]


def col_count(A, Cm: np.ndarray) -> np.ndarray:
    n, rp, ci, _ = _csr_args(A)
    cnt = np.zeros(n, np.int32)
    lib().or_col_count(n, rp, ci, np.ascontiguousarray(Cm, np.uint8), cnt)
    return cnt


def sym_graph(A, Cm: np.ndarray):
    n, rp, ci, _ = _csr_args(A)
    Cm = np.ascontiguousarray(Cm, np.uint8)
    Sptr = np.zeros(n + 1, np.int32)
    ns = lib().or_sym_graph(n, rp, ci, Cm, Sptr, None, 0)
    Scol = np.zeros(max(ns, 1), np.int32)
    lib().or_sym_graph(n, rp, ci, Cm, Sptr, Scol.ctypes.data, ns)
    return Sptr, Scol[:ns]


def mis_hash(seed: int, level: int, n: int) -> np.ndarray:
    L = lib()
    return np.array([L.or_mis_hash(seed, level, i) for i in range(n)], dtype=np.uint32)


def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x))


def pmis(Sptr, Scol, count, h, k: int = 2):
    """Alg. 2 with k max rounds per iteration: the roots of MIS(k) (Sec. 2.1.2)."""
    n = len(Sptr) - 1
    s = np.zeros(n, np.int8)
    Scol = np.ascontiguousarray(Scol, np.int32) if len(Scol) else np.zeros(1, np.int32)
    rounds = lib().or_pmis(n, np.ascontiguousarray(Sptr, np.int32), Scol, np.ascontiguousarray(count, np.int32),
                           np.ascontiguousarray(h, np.uint32), s, k)
    return s, rounds


def pmis2(Sptr, Scol, count, h):
    return pmis(Sptr, Scol, count, h, 2)


def aggregate(Sptr, Scol, count, h, s, k: int = 2):
    n = len(Sptr) - 1
    agg = np.zeros(n, np.int32)
    Scol = np.ascontiguousarray(Scol, np.int32) if len(Scol) else np.zeros(1, np.int32)
    nc = lib().or_aggregate(n, np.ascontiguousarray(Sptr, np.int32), Scol, np.ascontiguousarray(count, np.int32),
                            np.ascontiguousarray(h, np.uint32), np.ascontiguousarray(s, np.int8), agg, k)
    return agg, nc


def interp(agg, nc: int, B):
    n = len(agg)
    P = np.zeros(n)
    Bc = np.zeros(max(nc, 1))
    lib().or_interp(n, nc, np.ascontiguousarray(agg, np.int32), np.ascontiguousarray(B, np.float64), P, Bc)
    return P, Bc[:nc]


def galerkin(A, agg, nc: int, P=None):
    from paper_1403_1649_gb300.problems import CSR
    n, rp, ci, v = _csr_args(A)
    agg = np.ascontiguousarray(agg, np.int32)
    Pp = None if P is None else np.ascontiguousarray(P, np.float64)
    crp = np.zeros(nc + 1, np.int32)
    L = lib()
    cn = L.or_galerkin(n, rp, ci, v, nc, agg, None if Pp is None else Pp.ctypes.data, crp, None, None, 0)
    cci = np.zeros(max(cn, 1), np.int32)
    cval = np.zeros(max(cn, 1))
    L.or_galerkin(n, rp, ci, v, nc, agg, None if Pp is None else Pp.ctypes.data, crp, cci.ctypes.data,
                  cval.ctypes.data, cn)
    return CSR(nc, crp, cci[:cn], cval[:cn])


def rho_estimate(A, seed: int = 0, level: int = 0, m: int = 5, symmetric: bool = True):
    n, rp, ci, v = _csr_args(A)
    H = np.zeros(64)
    rho = lib().or_rho_estimate(n, rp, ci, v, seed, level, m, H.ctypes.data, 1 if symmetric else 0)
    mm = min(m, n)
    return rho, H[:mm * mm].reshape(mm, mm)


def sym_eig(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float64)
    w = np.zeros(a.shape[0])
    lib().or_sym_eig(a.shape[0], a.reshape(-1), w)
    return w


def cholesky(a: np.ndarray):
    L = np.ascontiguousarray(a, np.float64).copy()
    rc = lib().or_cholesky(L.shape[0], L.reshape(-1))
    return (L if rc == 0 else None)


def hess_rho(H: np.ndarray) -> float:
    """Largest |eigenvalue| of an upper Hessenberg matrix (shifted complex QR)."""
    H = np.ascontiguousarray(H, np.float64)
    return lib().or_hess_rho(H.shape[0], H.reshape(-1).copy())


def lu(a: np.ndarray):
    """In-place LU with partial pivoting: (LU, piv) or None if singular."""
    LU = np.ascontiguousarray(a, np.float64).copy()
    piv = np.zeros(LU.shape[0], np.int32)
    rc = lib().or_lu(LU.shape[0], LU.reshape(-1), piv)
    return (LU, piv) if rc == 0 else None


def lu_solve(LU: np.ndarray, piv: np.ndarray, b: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(b, np.float64).copy()
    lib().or_lu_solve(LU.shape[0], np.ascontiguousarray(LU).reshape(-1), piv, x)
    return x


def chol_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(b, np.float64).copy()
    lib().or_chol_solve(L.shape[0], np.ascontiguousarray(L).reshape(-1), x)
    return x


# ------------------------------------------------------------ learned smoother
NFEAT, HID, NOUT = 16, 64, 3
NPARAM = HID * NFEAT + HID + HID * HID + HID + NOUT * HID + NOUT


def features(A, level: int = 0) -> np.ndarray:
    n, rp, ci, v = _csr_args(A)
    f = np.zeros((n, NFEAT), np.float32)
    lib().or_features(n, rp, ci, v, level, f.reshape(-1))
    return f


def mlp_forward(w16: np.ndarray, feat: np.ndarray) -> np.ndarray:
    """FP32 MLP with FP16 weights; w16 holds binary16 bit patterns (uint16)."""
    w16 = np.ascontiguousarray(w16, np.uint16)
    feat = np.ascontiguousarray(feat, np.float32)
    out = np.zeros((feat.shape[0], NOUT), np.float32)
    lib().or_mlp_forward(feat.shape[0], w16, feat.reshape(-1), out.reshape(-1))
    return out


def mlp_backward(w: np.ndarray, feat: np.ndarray, dout: np.ndarray):
    """FP64 forward + backward: returns (dL/dparam, out) for L with dL/dout = dout."""
    feat = np.ascontiguousarray(feat, np.float32)
    dparam = np.zeros(NPARAM)
    out = np.zeros((feat.shape[0], NOUT))
    lib().or_mlp_backward(feat.shape[0], np.ascontiguousarray(w, np.float64), feat.reshape(-1),
                          np.ascontiguousarray(dout, np.float64).reshape(-1), dparam, out.ctypes.data)
    return dparam, out


# ------------------------------------------------------------ whole method
@dataclass
class Level:
    n: int
    nnz: int
    omega: float
    mis_rounds: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    agg: np.ndarray | None = None
    P: np.ndarray | None = None
    B: np.ndarray | None = None


def threads(omp: bool = True) -> int:
    """Host threads the solve stage of the given build uses."""
    return int(lib(omp).or_threads())


def default_params(**kw) -> ORParams:
    p = ORParams()
    lib().or_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Hierarchy:
    """Aggregation AMG hierarchy (Alg. 1) and its solve phase, on the CPU in FP64."""

    def __init__(self, A, omp: bool = False, **params):
        """omp=True: the OpenMP timing build (multi-threaded solve stage; the
        benchmark's CPU baseline), otherwise the single-threaded parity build."""
        self._L = lib(omp)
        self.params = default_params(**params)
        n, rp, ci, v = _csr_args(A)
        err = C.c_int32(0)
        self.h = self._L.or_setup(n, rp, ci, v, C.byref(self.params), C.byref(err))
        if not self.h:
            raise RuntimeError(f"oracle setup failed: {err.value}")
        self.n = n

    def subsystem(self, r0: int, r1: int) -> "Hierarchy":
        """The part of this hierarchy that belongs to rows [r0, r1) of level 0
        (one system of a block-diagonal batch), as a hierarchy of its own."""
        err = C.c_int32(0)
        ptr = self._L.or_subsystem(self.h, r0, r1, C.byref(err))
        if not ptr:
            raise ValueError(f"rows [{r0}, {r1}) do not form an independent block ({err.value})")
        sub = Hierarchy.__new__(Hierarchy)
        sub._L = self._L
        sub.params = self.params
        sub.h = ptr
        sub.n = r1 - r0
        return sub

    def __del__(self):
        if getattr(self, "h", None):
            self._L.or_free(self.h)
            self.h = None

    @property
    def nlevels(self) -> int:
        return self._L.or_nlevels(self.h)

    def level(self, k: int) -> Level:
        n, nnz, om, mr = C.c_int32(), C.c_int64(), C.c_double(), C.c_int32()
        self._L.or_level_info(self.h, k, C.byref(n), C.byref(nnz), C.byref(om), C.byref(mr))
        n, nnz = n.value, nnz.value
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        val = np.zeros(max(nnz, 1))
        last = k == self.nlevels - 1
        agg = None if last else np.zeros(n, np.int32)
        P = None if last else np.zeros(n)
        B = np.zeros(n)
        self._L.or_level_copy(self.h, k, rp.ctypes.data, ci.ctypes.data, val.ctypes.data,
                            None if last else agg.ctypes.data, None if last else P.ctypes.data, B.ctypes.data)
        return Level(n, nnz, om.value, mr.value, rp, ci[:nnz], val[:nnz], agg, P, B)

    def set_poly(self, k: int, coef: np.ndarray) -> None:
        coef = np.ascontiguousarray(coef, np.float64).reshape(-1)
        if self._L.or_set_poly(self.h, k, coef) != 0:
            raise ValueError("bad level for polynomial smoother")

    def cycle_trace(self) -> dict:
        """Per level: cycle visits, Alg. 5 coarse parts run, second inner steps (last solve/precond)."""
        nl = self.nlevels
        v, k, s2 = (np.zeros(nl, np.int64) for _ in range(3))
        self._L.or_cycle_trace(self.h, v.ctypes.data, k.ctypes.data, s2.ctypes.data)
        return {"visits": v, "kcalls": k, "second": s2}

    def precond(self, b: np.ndarray) -> np.ndarray:
        x = np.zeros(self.n)
        self._L.or_precond(self.h, np.ascontiguousarray(b, np.float64), x)
        return x

    def krylov2_probe(self, m: int, r: np.ndarray):
        n = self.level(m).n
        x, c, d = np.zeros(n), np.zeros(n), np.zeros(n)
        if self._L.or_krylov2_probe(self.h, m, np.ascontiguousarray(r, np.float64), x, c, d) != 0:
            raise ValueError("level has no K-cycle coarse part")
        return x, c, d

    def twogrid_loss(self, coef: np.ndarray, nvec: int = 4, seed: int = 0, grad: bool = True):
        """Two-grid error reduction of the polynomial pre-smoother (levels 0, 1)."""
        coef = np.ascontiguousarray(coef, np.float64).reshape(-1)
        d = np.zeros_like(coef) if grad else None
        L = self._L.or_twogrid_loss(self.h, coef, nvec, seed, None if d is None else d.ctypes.data)
        return L, (None if d is None else d.reshape(-1, 3))

    def solve(self, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-8, max_iter: int = 200):
        x = np.zeros(self.n) if x0 is None else np.ascontiguousarray(x0, np.float64).copy()
        hist = np.zeros(max_iter + 2)
        it = C.c_int32()
        fr = C.c_double()
        st = self._L.or_solve(self.h, np.ascontiguousarray(b, np.float64), x, tol, max_iter, C.byref(it), hist,
                            C.byref(fr))
        return x, {"status": st, "iters": it.value, "hist": hist[:it.value + 1].copy(), "relres": fr.value}
