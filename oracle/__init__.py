"""CPU oracle for the mixed-precision ILU(0)-preconditioned multi-component Krylov path.

TEST INFRASTRUCTURE.  This package is a plain, slow, single-threaded restatement of what the
method of Kouya (arXiv 2504.14498) computes: D/DD/TD/QD arithmetic, the mixed SpMV
(binary64 matrix times multi-component vector, Sec. 3), ILU(0) (Algorithm 1), the
substitutions (Algorithm 2) and the BiCG (Algorithm 3), CGS, BiCGSTAB and GPBiCG solvers.
Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may import it;
the CUDA library neither links nor calls it.

Layout conventions (shared with the library's C ABI by specification, not by code): a real
multi-component number is w doubles, leading component first; a complex one is 2w doubles
(real part then imaginary part); a vector is n*c*w doubles.

Parity pins for every function here live in tests/test_oracle_*.py.  Functions without a pin:
none at present.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

ILU_NONE, ILU_FP64, ILU_FP32, ILU_BF16, ILU_MP = -1, 0, 1, 2, 3
BICG, CGS, BICGSTAB, GPBICG = 0, 1, 2, 3
METHODS = {"bicg": BICG, "cgs": CGS, "bicgstab": BICGSTAB, "gpbicg": GPBICG}
ILUS = {"none": ILU_NONE, "fp64": ILU_FP64, "fp32": ILU_FP32, "bf16": ILU_BF16, "mp": ILU_MP}
STATUS = {0: "OK", 1: "MAXIT", 2: "BREAKDOWN", 3: "ZERO_PIVOT", 4: "MISSING_DIAG", 5: "NAN", 6: "INVALID_ARG"}

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I = ctypes.c_int
_D = ctypes.c_double
_IP = ctypes.POINTER(ctypes.c_int)
_DP = ctypes.POINTER(ctypes.c_double)


_lib_p = None


def lib_p():
    """The paper-like "_p" build (SpMV, vector updates and inner products on all host threads),
    or None where OpenMP is unavailable.  Used only by the benchmark's CPU baseline."""
    global _lib_p
    if _lib_p is None:
        path = _build.build_p()
        if path is None:
            return None
        _lib_p = _declare(ctypes.CDLL(path))
    return _lib_p


def threads_p(k=0):
    """Threads of the "_p" build (k > 0 sets them); None without it."""
    L = lib_p()
    return None if L is None else L.orc_threads(int(k))


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(_build.build()))
    return _lib


def _declare(L):
    L.orc_two_sum.argtypes = [_D, _D, _f64p]
    L.orc_two_prod.argtypes = [_D, _D, _f64p]
    L.orc_mp_op.argtypes = [_I, _I, _f64p, _f64p, _f64p]
    L.orc_spmv.argtypes = [_I, _i32p, _i32p, _f64p, _I, _I, _f64p, _f64p]
    L.orc_spmv_mm.argtypes = [_I, _i32p, _i32p, _f64p, _I, _I, _f64p, _f64p]
    L.orc_dot.argtypes = [_I, _I, _I, _f64p, _f64p, _f64p]
    L.orc_check_pattern.argtypes = [_I, _i32p, _i32p, ctypes.c_void_p, _IP]
    L.orc_check_pattern.restype = _I
    L.orc_ilu0.argtypes = [_I, _i32p, _i32p, _f64p, _I, _I, _f64p, _IP]
    L.orc_ilu0.restype = _I
    L.orc_ilu0_mp.argtypes = [_I, _i32p, _i32p, _f64p, _I, _I, _f64p, _IP]
    L.orc_ilu0_mp.restype = _I
    L.orc_precond.argtypes = [_I, _i32p, _i32p, _f64p, _I, _I, _I, _I, _f64p, _f64p]
    L.orc_krylov.argtypes = [_I, _I, _i32p, _i32p, _f64p, _I, _I, _I, ctypes.c_void_p, _f64p, _f64p,
                             _D, _D, _I, _I, _f64p, _IP, _DP, _I, ctypes.c_void_p, _IP]
    L.orc_krylov_hooks.argtypes = [_I, _I, _i32p, _i32p, _f64p, _I, _I, _I, ctypes.c_void_p, _f64p, _f64p,
                                   _D, _D, _I, _I, _f64p, _IP, _DP, ctypes.c_void_p, ctypes.c_void_p,
                                   _I, _f64p, _IP]
    L.orc_krylov.restype = _I
    L.orc_threads.argtypes = [_I]
    L.orc_threads.restype = _I
    return L


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def two_sum(a, b):
    out = np.zeros(2)
    lib().orc_two_sum(float(a), float(b), out)
    return out


def two_prod(a, b):
    out = np.zeros(2)
    lib().orc_two_prod(float(a), float(b), out)
    return out


_OPS = {"add": 0, "sub": 1, "mul": 2, "mul_d": 3, "div": 4, "div_d": 5, "sqrt": 6}


def mp_op(op, w, a, b=None):
    """One real multi-component operation; a, b are length-w component arrays (b[0] is the
    binary64 operand for mul_d / div_d)."""
    a = _c(np.resize(np.asarray(a, dtype=np.float64), 4), np.float64)
    b = _c(np.resize(np.asarray(b if b is not None else np.zeros(w), dtype=np.float64), 4), np.float64)
    out = np.zeros(4)
    lib().orc_mp_op(_OPS[op], w, a, b, out)
    return out[:w]


def spmv(A, x, w, c=1, mp_matrix=False):
    """y = A x; A = (n, row_ptr, col, val) with val interleaved re,im when c == 2.
    mp_matrix: the matrix entries promoted to w components (the rows without "_d")."""
    n, rp, ci, val = A
    y = np.zeros(n * c * w)
    f = lib().orc_spmv_mm if mp_matrix else lib().orc_spmv
    f(n, _c(rp, np.int32), _c(ci, np.int32), _c(val, np.float64), c, w, _c(x, np.float64), y)
    return y


def dot(a, b, n, w, c=1):
    """<a, b> = sum_i conj(a_i) b_i, sequential left-to-right accumulation."""
    out = np.zeros(c * w)
    lib().orc_dot(n, c, w, _c(a, np.float64), _c(b, np.float64), out)
    return out


def check_pattern(A):
    n, rp, ci, _ = A
    fr = ctypes.c_int(-1)
    st = lib().orc_check_pattern(n, _c(rp, np.int32), _c(ci, np.int32), None, ctypes.byref(fr))
    return st, fr.value


def ilu0(A, prec="fp64", c=1, w=1):
    """ILU(0) factor on A's pattern (Algorithm 1); returns (status, factor values, fail_row).
    prec 'mp': the factor in w-component arithmetic (nnz * c * w values)."""
    n, rp, ci, val = A
    fr = ctypes.c_int(-1)
    if prec == "mp":
        fac = np.zeros(len(ci) * c * w)
        st = lib().orc_ilu0_mp(n, _c(rp, np.int32), _c(ci, np.int32), _c(val, np.float64), c, w, fac,
                               ctypes.byref(fr))
        return st, fac, fr.value
    fac = np.zeros(len(ci) * c)
    st = lib().orc_ilu0(n, _c(rp, np.int32), _c(ci, np.int32), _c(val, np.float64), c, ILUS[prec], fac, ctypes.byref(fr))
    return st, fac, fr.value


def precond(A, fac, r, w, prec="fp64", c=1, trans=False):
    """z = M^-1 r (trans=False) or M^-H r (trans=True), Algorithm 2."""
    n, rp, ci, _ = A
    z = np.zeros(n * c * w)
    lib().orc_precond(n, _c(rp, np.int32), _c(ci, np.int32), _c(fac, np.float64), c, w, ILUS[prec], int(trans),
                      _c(r, np.float64), z)
    return z


TRUE_RES_PERIOD = 50  # default period of the true-residual check (0: none)


def krylov(method, A, b, w, c=1, ilu="none", fac=None, x0=None, tol_rel=1e-25, tol_abs=0.0, maxit=1000,
           force_eta0=False, mp_matrix=False, shadow=None, trace=False, true_res_period=TRUE_RES_PERIOD,
           parallel=False):
    """Run one solve; returns dict(status, iters, x, hist, relres_true, hist_true, replacements).
    mp_matrix: every SpMV with the matrix promoted to w components (the rows without "_d").
    true_res_period: P > 0 recomputes b - A x every P iterations and when the recursive residual
    passes the stopping test, replacing r when the true norm is above 10x the target (then a
    passed test is withdrawn); hist_true[k] is that norm at the checked iterations, NaN elsewhere.
    Test hooks: shadow, the initial shadow residual instead of r0; trace, also return "trace"
    (per iteration the normalised inner products that exact arithmetic makes zero).
    parallel: run on the "_p" build (benchmark baseline only; its inner products are summed per
    thread range, so its bits differ from the plain oracle's)."""
    n, rp, ci, val = A
    x = np.zeros(n * c * w) if x0 is None else _c(x0, np.float64).copy()
    hist = np.zeros(maxit + 2)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    facp = None
    if ILUS[ilu] >= 0:
        if fac is None:
            st, fac, fr = ilu0(A, ilu, c, w)
            if st != 0:
                return {"status": STATUS[st], "iters": 0, "x": x, "hist": hist[:1], "relres_true": float("nan"),
                        "fail_row": fr}
        fac = _c(fac, np.float64)
        facp = fac.ctypes.data_as(ctypes.c_void_p)
    sh = None if shadow is None else _c(shadow, np.float64)
    tr = np.zeros(2 * (maxit + 2)) if trace else None
    htrue = np.full(maxit + 2, np.nan)
    nrep = ctypes.c_int(0)
    L = lib_p() if parallel else lib()
    if L is None:
        raise RuntimeError("the OpenMP build of the oracle is unavailable")
    st = L.orc_krylov_hooks(METHODS[method], n, _c(rp, np.int32), _c(ci, np.int32), _c(val, np.float64), c, w,
                                ILUS[ilu], facp, _c(b, np.float64), x, float(tol_rel), float(tol_abs), int(maxit),
                                (1 if force_eta0 else 0) | (2 if mp_matrix else 0), hist, ctypes.byref(it),
                                ctypes.byref(rr), None if sh is None else sh.ctypes.data_as(ctypes.c_void_p),
                                None if tr is None else tr.ctypes.data_as(ctypes.c_void_p), int(true_res_period),
                                htrue, ctypes.byref(nrep))
    out = {"status": STATUS[st], "iters": it.value, "x": x, "hist": hist[: it.value + 1].copy(),
           "relres_true": rr.value, "hist_true": htrue[: it.value + 1].copy(), "replacements": nrep.value}
    if trace:
        out["trace"] = tr.reshape(-1, 2)[1: it.value + 1].copy()
    return out
