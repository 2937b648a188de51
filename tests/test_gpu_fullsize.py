"""GPU parity at the workloads' full sizes, in the launch configuration the benchmark times.

  * 2-D convection-diffusion 64 x 64 (N = 4096), cell Peclet 10: every method with D, DD and QD
    vectors and a binary64 ILU(0), to convergence, against the oracle's complete runs.
  * 3-D convection-diffusion 128^3 (N = 2,097,152, nnz = 14,581,760): DD SpMV, ILU(0) in
    binary64 / binary32 / bfloat16 and M^-1 compared in full; QD SpMV on sampled rows; the first
    DD BiCGSTAB iterations (residual history and iterate) with each factor precision.
  * shifted-Laplacian Helmholtz 1024 x 1024 complex (N = 1,048,576, nnz = 5,238,784): complex DD
    SpMV, complex ILU(0) in binary64 / binary32, M^-1 and M^-H, and the first iterations of
    complex DD BiCGSTAB and BiCG.
Bars as in test_gpu_parity: bitwise for the D / DD SpMV, the factors and the substitutions (the
GPU follows the oracle's operation order), within 2^-200 of sum |a||x| per row for QD; solves
within the stated bars of tests/_bars.py (the inner products differ in summation order).
"""
import numpy as np
import pytest
import torch

import _bars
import oracle
from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def cube():
    A_t, meta = inputs.convdiff3d(128)
    assert A_t[0] == 2097152 and len(A_t[2]) == 14581760
    return A_t, _lib.Matrix.from_tuple(A_t)


@pytest.fixture(scope="module")
def helm():
    A_t = inputs.helmholtz2d(1024, k=20 * np.pi)
    assert A_t[0] == 1048576 and len(A_t[2]) == 5238784
    return A_t, _lib.Matrix.from_tuple(A_t, is_complex=True)


def _rows(A_t, rows):
    n, rp, ci, val = A_t
    lens = rp[rows + 1] - rp[rows]
    sub_rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    return (len(rows), sub_rp, ci[idx], val[idx])


# ---- 64 x 64 2-D: complete solves ---------------------------------------------------------------
@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
@pytest.mark.parametrize("w,tol", [(1, 1e-13), (2, 1e-25), (4, 1e-25)])
def test_convdiff2d_64_complete_solves(method, w, tol):
    A_t = inputs.convdiff2d(64, pe=10.0)
    n = A_t[0]
    assert n == 4096 and len(A_t[2]) == 20224
    xs = inputs.ones(n, w)
    A = _lib.Matrix.from_tuple(A_t)
    b = _lib.spmv_mp(A, dev(xs), w)
    b_ref = oracle.spmv(A_t, xs, w)
    M = _lib.ILU0(A, "fp64")
    out = _lib.krylov_solve(method, w, A, M, b, tol_rel=tol, maxit=2000)
    ref = oracle.krylov(method, A_t, b_ref, w, ilu="fp64", tol_rel=tol, maxit=2000)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, "fp64", w, tol)
    xe = host(out["x"]).reshape(n, w)
    err = np.max(np.abs((xe[:, 0] - 1.0) + xe[:, 1:].sum(axis=1)))
    assert err < {1: 1e-9, 2: 1e-20, 4: 1e-20}[w]


# ---- 128^3 3-D ----------------------------------------------------------------------------------
def test_cube_spmv_dd_full(cube):
    A_t, A = cube
    x = inputs.random_vector(A_t[0], 2, 1, seed=301)
    assert np.array_equal(host(_lib.spmv_mp(A, dev(x), 2)), oracle.spmv(A_t, x, 2))


def test_cube_spmv_qd_sampled(cube):
    A_t, A = cube
    n = A_t[0]
    x = inputs.random_vector(n, 4, 1, seed=302)
    y = host(_lib.spmv_mp(A, dev(x), 4)).reshape(n, 4)
    rows = np.unique(np.concatenate([np.arange(0, n, 1009), [n - 1]]))
    sub = _rows(A_t, rows)
    ref = oracle.spmv(sub, x, 4).reshape(len(rows), 4)
    X = np.abs(x.reshape(n, 4)[:, 0])
    mag = np.add.reduceat(np.abs(sub[3]) * X[sub[2]], sub[1][:-1])
    err = np.abs(_bars.mp_diff(y[rows], ref, 4))
    assert np.all(err <= 2.0 ** -200 * mag * 4)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_cube_ilu_and_precond_full(cube, prec):
    A_t, A = cube
    n = A_t[0]
    M = _lib.ILU0(A, prec)
    st, fac, _ = oracle.ilu0(A_t, prec)
    assert st == 0
    assert np.array_equal(host(M.values()), fac)
    r = inputs.random_vector(n, 2, 1, seed=303)
    assert np.array_equal(host(M.apply(dev(r), 2)), oracle.precond(A_t, fac, r, 2, prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cube_bicgstab_first_iterations(cube, prec):
    A_t, A = cube
    n, w, its = A_t[0], 2, 2
    xs = inputs.ones(n, w)
    b = _lib.spmv_mp(A, dev(xs), w)
    b_ref = oracle.spmv(A_t, xs, w)
    assert np.array_equal(host(b), b_ref)
    out = _lib.krylov_solve("bicgstab", w, A, _lib.ILU0(A, prec), b, tol_rel=1e-25, maxit=its)
    ref = oracle.krylov("bicgstab", A_t, b_ref, w, ilu=prec, tol_rel=1e-25, maxit=its)
    assert out["status"] == ref["status"] == "MAXIT"
    assert _bars.check_band(out["hist"], ref["hist"], _bars.band_floor(prec, w)) == its + 1
    assert _bars.rel_error(host(out["x"]), ref["x"], n, 1, w) <= 1e-24


# ---- 1024^2 complex Helmholtz -------------------------------------------------------------------
def test_helmholtz_spmv_full(helm):
    A_t, A = helm
    x = inputs.random_vector(A_t[0], 2, 2, seed=311)
    assert np.array_equal(host(_lib.spmv_mp(A, dev(x), 2)), oracle.spmv(A_t, x, 2, 2))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_helmholtz_ilu_and_precond_full(helm, prec):
    A_t, A = helm
    n = A_t[0]
    M = _lib.ILU0(A, prec)
    st, fac, _ = oracle.ilu0(A_t, prec, 2)
    assert st == 0
    assert np.array_equal(host(M.values()), fac)
    r = inputs.random_vector(n, 2, 2, seed=312)
    for trans in (False, True):
        assert np.array_equal(host(M.apply(dev(r), 2, trans)), oracle.precond(A_t, fac, r, 2, prec, 2, trans))


@pytest.mark.parametrize("method", ["bicgstab", "bicg"])
def test_helmholtz_first_iterations(helm, method):
    A_t, A = helm
    n, w, its = A_t[0], 2, 2
    b_h = inputs.normal_rhs(n, w, 2)
    out = _lib.krylov_solve(method, w, A, _lib.ILU0(A, "fp64"), dev(b_h), tol_rel=1e-25, maxit=its)
    ref = oracle.krylov(method, A_t, b_h, w, 2, ilu="fp64", tol_rel=1e-25, maxit=its)
    assert out["status"] == ref["status"] == "MAXIT"
    assert _bars.check_band(out["hist"], ref["hist"], _bars.band_floor("fp64", w)) == its + 1
    assert _bars.rel_error(host(out["x"]), ref["x"], n, 2, w) <= 1e-24
