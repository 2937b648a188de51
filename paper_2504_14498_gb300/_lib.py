"""ctypes binding of libmpk.so (include/mpk.h).  Argument marshalling only: every step of the
solver runs in the library's CUDA kernels; torch supplies device memory and the stream.

There is no fallback: if libmpk.so is missing or cannot be loaded, every call raises.
"""
import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpk.so")

STATUS = {0: "OK", 1: "MAXIT", 2: "BREAKDOWN", 3: "ZERO_PIVOT", 4: "MISSING_DIAG", 5: "NAN", 6: "INVALID_ARG",
          7: "CUDA_ERROR", 8: "TIMEOUT", 9: "NOT_IMPLEMENTED"}
METHODS = {"bicg": 0, "cgs": 1, "bicgstab": 2, "gpbicg": 3}
ILUS = {"none": -1, "fp64": 0, "fp32": 1, "bf16": 2, "mp": 3}
FLAG_ETA0, FLAG_MP_MATRIX = 1, 2  # mpk_opts.flags bits


class MpkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = STATUS.get(status, status)


class CsrDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("is_complex", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("tol_rel", ctypes.c_double), ("tol_abs", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("flags", ctypes.c_int32), ("true_res_period", ctypes.c_int32),
                ("hist_dev", ctypes.c_void_p), ("hist_true_dev", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("fail_row", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("res0", ctypes.c_double), ("relres_rec", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("ms_solve", ctypes.c_float), ("hermitian", ctypes.c_int32),
                ("replacements", ctypes.c_int32)]


_lib = None

# (name, restype, argtypes) of every entry point declared in include/mpk.h
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = [
    ("mpk_version", _I, []),
    ("mpk_last_error", ctypes.c_char_p, []),
    ("mpk_kernel_launches", ctypes.c_uint64, []),
    ("mpk_spmv_mp", _I, [ctypes.POINTER(CsrDesc), _I, _VP, _VP, _VP]),
    ("mpk_spmv_mp_matrix", _I, [ctypes.POINTER(CsrDesc), _I, _VP, _VP, _VP]),
    ("mpk_dot", _I, [_I, _I, _I, _VP, _VP, _VP, _VP]),
    ("mpk_dot_noalloc", _I, [_I, _I, _I, _VP, _VP, _VP, _VP]),
    ("mpk_mp_op", _I, [_I, _I, _I, _VP, _VP, _VP, _VP]),
    ("mpk_probe_notify_ns", _I, [_I, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I), _VP]),
    ("mpk_ilu0_factor", _I, [ctypes.POINTER(CsrDesc), _I, ctypes.POINTER(_VP), ctypes.POINTER(_I), _VP]),
    ("mpk_ilu0_factor_mp", _I, [ctypes.POINTER(CsrDesc), _I, ctypes.POINTER(_VP), ctypes.POINTER(_I), _VP]),
    ("mpk_ilu0_values", _I, [_VP, _VP, _VP]),
    ("mpk_ilu0_prec", _I, [_VP]),
    ("mpk_ilu0_width", _I, [_VP]),
    ("mpk_ilu0_schedule", _I, [_VP, ctypes.POINTER(_I)]),
    ("mpk_ilu0_polling", _I, [_VP]),
    ("mpk_ilu0_levels", _I, [_VP, _I, ctypes.POINTER(_I), _VP, _VP]),
    ("mpk_ilu0_test_withhold", _I, [_VP, _I]),
    ("mpk_ilu0_destroy", None, [_VP]),
    ("mpk_precond_apply", _I, [_VP, _I, _I, _VP, _VP, _VP]),
    ("mpk_krylov_solve", _I, [_I, _I, ctypes.POINTER(CsrDesc), _VP, _VP, _VP, ctypes.POINTER(Opts),
                              ctypes.POINTER(Info), _VP]),
    ("mpk_solve_host", _I, [_I, _I, _I, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP,
                            ctypes.POINTER(Opts), ctypes.POINTER(Info)]),
    ("mpk_krylov_solve_batched", _I, [_I, _I, ctypes.POINTER(CsrDesc), _I, _VP, _VP, _VP, _VP, _VP,
                                      ctypes.POINTER(Opts), ctypes.POINTER(Info), _VP]),
    ("mpk_gnn_nparams", _I, []),
    ("mpk_gnn_workspace_bytes", ctypes.c_size_t, [_I, _I, _I, _I]),
    ("mpk_gnn_forward", _I, [ctypes.POINTER(CsrDesc), _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("mpk_gnn_loss", _I, [ctypes.POINTER(CsrDesc), _VP, _VP, _I, _VP, _I, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("mpk_gnn_loss_precond", _I, [ctypes.POINTER(CsrDesc), _VP, _VP, _I, _VP, _I, _VP, _VP, _VP, _VP,
                                  ctypes.c_size_t, _VP]),
    ("mpk_gnn_backward", _I, [ctypes.POINTER(CsrDesc), _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    ("mpk_gnn_adam", _I, [_I, _VP, _VP, _VP, _VP, ctypes.c_float, _I, _VP]),
    ("mpk_ilu0_correct", _I, [_VP, _VP, _VP]),
]


def lib():
    """Load libmpk.so (built by paper_2504_14498_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmpk.so is not built (run paper_2504_14498_gb300.build.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels launched by libmpk so far in this process."""
    return int(lib().mpk_kernel_launches())


def _check(st):
    if st != 0:
        raise MpkError(st, lib().mpk_last_error().decode())
    return st


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, numel=None, dtype=None, name="buffer"):
    """Device pointer of a tensor the library reads or writes.  The C functions take raw pointers
    and sizes, so a host tensor, a strided view, a narrower dtype or a short buffer is refused
    here, before any call (MPK_INVALID_ARG semantics, as ValueError)."""
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s: expected a torch tensor, got %s" % (name, type(t).__name__))
    if t.device.type != "cuda":
        raise ValueError("%s: the library needs device memory (a CUDA tensor), got %s" % (name, t.device))
    if not t.is_contiguous():
        raise ValueError("%s: must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s: expected %s, got %s" % (name, dtype, t.dtype))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s: needs at least %d elements, has %d" % (name, numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _vec(t, numel, name):
    """A multi-component vector argument: float64, on the device, contiguous, numel doubles."""
    return _ptr(t, numel, torch.float64, name)


class Matrix:
    """Device CSR matrix (torch tensors) with the C descriptor."""

    def __init__(self, n, row_ptr, col_idx, val, is_complex=False, device="cuda"):
        self.n = int(n)
        self.row_ptr = torch.as_tensor(np.asarray(row_ptr, dtype=np.int32), device=device)
        self.col_idx = torch.as_tensor(np.asarray(col_idx, dtype=np.int32), device=device)
        self.val = torch.as_tensor(np.asarray(val, dtype=np.float64), device=device)
        self.is_complex = bool(is_complex)
        self.nnz = int(self.col_idx.numel())
        self.cp = 2 if is_complex else 1
        self.desc = CsrDesc(self.n, self.nnz, self.row_ptr.data_ptr(), self.col_idx.data_ptr(),
                            self.val.data_ptr(), int(self.is_complex))

    @classmethod
    def from_tuple(cls, A, is_complex=False, device="cuda"):
        n, rp, ci, val = A
        return cls(n, rp, ci, val, is_complex, device)


def spmv_mp(A: Matrix, x: torch.Tensor, w: int, y: torch.Tensor = None, mp_matrix=False) -> torch.Tensor:
    """y = A x with w-component vectors (n*c*w doubles); mp_matrix: A's entries promoted to w
    components (the rows without "_d")."""
    m = A.n * A.cp * w
    if y is None:
        y = torch.empty(m, dtype=torch.float64, device=x.device)
    px, py = _vec(x, m, "x"), _vec(y, m, "y")
    f = lib().mpk_spmv_mp_matrix if mp_matrix else lib().mpk_spmv_mp
    _check(f(ctypes.byref(A.desc), w, px, py, _stream()))
    return y


def dot(a: torch.Tensor, b: torch.Tensor, n: int, w: int, is_complex=False) -> torch.Tensor:
    """<a, b> = sum conj(a_i) b_i; returns a device tensor of c*w doubles."""
    c = 2 if is_complex else 1
    out = torch.empty(c * w, dtype=torch.float64, device=a.device)
    m = n * c * w
    _check(lib().mpk_dot(n, int(is_complex), w, _vec(a, m, "a"), _vec(b, m, "b"), _vec(out, c * w, "out"),
                         _stream()))
    return out


def dot_noalloc(a: torch.Tensor, b: torch.Tensor, n: int, w: int, is_complex=False, out: torch.Tensor = None):
    """Same as dot(), for callers that must not let the library allocate device memory: the
    reduction scratch is a fixed array inside the library (n <= MPK_DOT_NOALLOC_MAX_N).  `out`
    may be preallocated by the caller (c*w doubles)."""
    c = 2 if is_complex else 1
    if out is None:
        out = torch.empty(c * w, dtype=torch.float64, device=a.device)
    m = n * c * w
    _check(lib().mpk_dot_noalloc(n, int(is_complex), w, _vec(a, m, "a"), _vec(b, m, "b"), _vec(out, c * w, "out"),
                                 _stream()))
    return out


def probe_notify_ns(rounds=2000, partner=1, with_sms=False):
    """One-way cross-SM notification latency in ns between block 0 and block `partner` of a grid
    with one block per SM (mpk_probe_notify_ns); with_sms: also the two SM ids."""
    v = ctypes.c_double(0.0)
    sms = (_I * 2)()
    _check(lib().mpk_probe_notify_ns(int(rounds), int(partner), ctypes.byref(v), sms, _stream()))
    return (v.value, (sms[0], sms[1])) if with_sms else v.value


MP_OPS = {"add": 0, "sub": 1, "mul": 2, "mul_fp": 3, "div": 4, "div_fp": 5, "sqrt": 6}


def mp_op(op: str, w: int, a: torch.Tensor, b: torch.Tensor = None, out: torch.Tensor = None) -> torch.Tensor:
    """Elementwise real w-component arithmetic (mpk_mp_op): a, b hold n*w doubles (entries of w
    components); mul_fp / div_fp use each b entry's leading component as the binary64 operand."""
    m = a.numel()
    if m % w:
        raise ValueError("a must hold whole w-component entries")
    if out is None:
        out = torch.empty_like(a)
    pb = None if b is None else _vec(b, m, "b")
    _check(lib().mpk_mp_op(MP_OPS[op], w, m // w, _vec(a, m, "a"), pb, _vec(out, m, "out"), _stream()))
    return out


class ILU0:
    """ILU(0) handle (Algorithm 1) in 'fp64', 'fp32' or 'bf16', or in w-component arithmetic
    ('mp', with w: the factor of the rows without "_d", serving solves with the same w)."""

    def __init__(self, A: Matrix, prec="fp64", w: int = None):
        self.A = A
        self.prec = prec
        self.w = w if prec == "mp" else 1
        h = ctypes.c_void_p()
        fr = ctypes.c_int(-1)
        if prec == "mp":
            if w is None:
                raise ValueError("prec 'mp' needs the component count w")
            st = lib().mpk_ilu0_factor_mp(ctypes.byref(A.desc), int(w), ctypes.byref(h), ctypes.byref(fr), _stream())
        else:
            st = lib().mpk_ilu0_factor(ctypes.byref(A.desc), ILUS[prec], ctypes.byref(h), ctypes.byref(fr), _stream())
        self.fail_row = fr.value
        if st != 0:
            raise MpkError(st, lib().mpk_last_error().decode() + " (row %d)" % fr.value)
        self.handle = h

    def schedule(self):
        """(schedule, warps per SM) of the substitutions: 'static', 'owner', 'cluster8' or
        'cluster16'."""
        wpb = ctypes.c_int(0)
        sc = lib().mpk_ilu0_schedule(self.handle, ctypes.byref(wpb))
        return ("static", "owner", "cluster8", "cluster16")[sc], wpb.value

    def polling(self):
        """Dependency polling of the substitutions: 'lane0', 'all' or 'allsleep'."""
        return ("lane0", "all", "allsleep")[lib().mpk_ilu0_polling(self.handle)]

    def levels(self, tri: int):
        """(number of levels, level of every row as a device int32 tensor) of L~ (tri 0) or U~
        (tri 1)."""
        nl = ctypes.c_int(0)
        depth = torch.empty(self.A.n, dtype=torch.int32, device="cuda")
        _check(lib().mpk_ilu0_levels(self.handle, int(tri), ctypes.byref(nl), _ptr(depth, self.A.n, torch.int32,
                                                                                 "depth"), _stream()))
        return nl.value, depth

    def test_withhold(self, row: int):
        """Testing aid: leave `row` unpublished in the substitutions (-1: none)."""
        _check(lib().mpk_ilu0_test_withhold(self.handle, int(row)))

    def values(self) -> torch.Tensor:
        out = torch.empty(self.A.nnz * self.A.cp * self.w, dtype=torch.float64, device="cuda")
        _check(lib().mpk_ilu0_values(self.handle, _ptr(out), _stream()))
        return out

    def apply(self, r: torch.Tensor, w: int, trans=False, z: torch.Tensor = None) -> torch.Tensor:
        if z is None:
            z = torch.empty_like(r)
        m = self.A.n * self.A.cp * w
        _check(lib().mpk_precond_apply(self.handle, w, int(trans), _vec(r, m, "r"), _vec(z, m, "z"), _stream()))
        return z

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().mpk_ilu0_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TRUE_RES_PERIOD = 50  # default period of the true-residual check (mpk_opts.true_res_period)


def krylov_solve(method, w, A: Matrix, M: ILU0, b: torch.Tensor, x0: torch.Tensor = None, tol_rel=1e-25,
                 tol_abs=0.0, maxit=1000, check_every=25, history=True, force_eta0=False, mp_matrix=False,
                 true_res_period=TRUE_RES_PERIOD):
    """Solve A x = b; returns dict(status, iters, x, hist, hist_true, replacements, res0, relres_rec,
    relres_true, ms, graph, hermitian).  mp_matrix: every SpMV with A's entries promoted to w
    components.  true_res_period: residual replacement period (0: off); hist_true holds
    ||b - A x_k|| at the checked iterations and NaN elsewhere."""
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    hist = torch.full((maxit + 1,), float("nan"), dtype=torch.float64, device=b.device) if history else None
    htrue = torch.full((maxit + 1,), float("nan"), dtype=torch.float64, device=b.device) if history else None
    flags = (FLAG_ETA0 if force_eta0 else 0) | (FLAG_MP_MATRIX if mp_matrix else 0)
    opts = Opts(float(tol_rel), float(tol_abs), int(maxit), int(check_every), flags, int(true_res_period),
                hist.data_ptr() if history else None, htrue.data_ptr() if history else None)
    info = Info()
    m = A.n * A.cp * w
    pb, px = _vec(b, m, "b"), _vec(x, m, "x0")
    st = lib().mpk_krylov_solve(METHODS[method], w, ctypes.byref(A.desc), M.handle if M is not None else None,
                                pb, px, ctypes.byref(opts), ctypes.byref(info), _stream())
    if st not in (0, 1, 2, 5):
        raise MpkError(st, lib().mpk_last_error().decode())
    h = hist[: info.iters + 1].cpu().numpy() if history else None
    ht = htrue[: info.iters + 1].cpu().numpy() if history else None
    return {"status": STATUS[info.status], "iters": info.iters, "x": x, "hist": h, "hist_true": ht,
            "replacements": info.replacements, "res0": info.res0, "relres_rec": info.relres_rec,
            "relres_true": info.relres_true, "ms": info.ms_solve, "graph": bool(info.graph),
            "hermitian": bool(info.hermitian)}


def krylov_solve_batched(method, w, A: Matrix, sys_rows, M: ILU0, b: torch.Tensor, x0: torch.Tensor = None,
                         tol_rel=1e-25, tol_abs=0.0, maxit=1000, check_every=25, history=False, mp_matrix=False,
                         true_res_period=TRUE_RES_PERIOD):
    """Solve the nsys independent systems of the block-diagonal A (system s: rows sys_rows[s] ..
    sys_rows[s+1]-1) together; returns dict(status, x, per-system arrays: statuses, iters, res0,
    relres_rec, relres_true, replacements, and hist, hist_true (nsys x (maxit+1)) when asked)."""
    rows = np.ascontiguousarray(np.asarray(sys_rows, dtype=np.int32))
    nsys = len(rows) - 1
    rows_dev = torch.as_tensor(rows, device=b.device)
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    hist = torch.full((nsys, maxit + 1), float("nan"), dtype=torch.float64, device=b.device) if history else None
    htrue = torch.full((nsys, maxit + 1), float("nan"), dtype=torch.float64, device=b.device) if history else None
    opts = Opts(float(tol_rel), float(tol_abs), int(maxit), int(check_every), FLAG_MP_MATRIX if mp_matrix else 0,
                int(true_res_period), hist.data_ptr() if history else None, htrue.data_ptr() if history else None)
    infos = (Info * nsys)()
    m = A.n * A.cp * w
    pb, px = _vec(b, m, "b"), _vec(x, m, "x0")
    st = lib().mpk_krylov_solve_batched(METHODS[method], w, ctypes.byref(A.desc), nsys, rows.ctypes.data,
                                        _ptr(rows_dev), M.handle if M is not None else None, pb, px,
                                        ctypes.byref(opts), infos, _stream())
    if st not in (0, 1, 2, 5):
        raise MpkError(st, lib().mpk_last_error().decode())
    out = {"status": STATUS[st], "x": x,
           "statuses": [STATUS[i.status] for i in infos],
           "iters": np.array([i.iters for i in infos]), "res0": np.array([i.res0 for i in infos]),
           "relres_rec": np.array([i.relres_rec for i in infos]),
           "relres_true": np.array([i.relres_true for i in infos]), "ms": infos[0].ms_solve,
           "replacements": np.array([i.replacements for i in infos]), "graph": bool(infos[0].graph)}
    if history:
        h = hist.cpu().numpy()
        out["hist"] = [h[s_, : out["iters"][s_] + 1] for s_ in range(nsys)]
        ht = htrue.cpu().numpy()
        out["hist_true"] = [ht[s_, : out["iters"][s_] + 1] for s_ in range(nsys)]
    return out


def solve_host(method, w, prec, A_tuple, b: np.ndarray, x0: np.ndarray = None, is_complex=False, tol_rel=1e-25,
               tol_abs=0.0, maxit=1000, check_every=25, true_res_period=TRUE_RES_PERIOD, x_inplace=False):
    """End to end from host arrays: H2D copies, ILU(0), solve, D2H of x inside one C call.
    x_inplace: x0 (float64, contiguous) is itself the in/out buffer of x (no host copy of it; pass
    page-locked arrays for full-speed copies)."""
    n, rp, ci, val = A_tuple
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if x_inplace:
        if x0 is None or x0.dtype != np.float64 or not x0.flags["C_CONTIGUOUS"]:
            raise ValueError("x_inplace needs x0 as a contiguous float64 array")
        x = x0
    else:
        x = np.zeros_like(b) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
    opts = Opts(float(tol_rel), float(tol_abs), int(maxit), int(check_every), 0, int(true_res_period), None, None)
    info = Info()
    st = lib().mpk_solve_host(METHODS[method], w, ILUS[prec], n, int(is_complex), rp.ctypes.data, ci.ctypes.data,
                              val.ctypes.data, b.ctypes.data, x.ctypes.data, ctypes.byref(opts), ctypes.byref(info))
    if st not in (0, 1, 2, 5):
        raise MpkError(st, lib().mpk_last_error().decode())
    return {"status": STATUS[info.status], "iters": info.iters, "x": x, "relres_true": info.relres_true,
            "replacements": info.replacements, "ms": info.ms_solve}
