"""The paper-scale stand-ins reproduce the shape of Tables 1 and 2 in the oracle (Sec. 4): without
ILU(0) the iteration stops at 3n without reaching 1e-13 (eps_a = 1e-100); with ILU(0) it converges,
in about ten iterations on the real matrix and in hundreds on the complex one; the plain rows and
the "_d" rows need the same iterations to within a few."""
import numpy as np
import pytest

import oracle
from paper_2504_14498_gb300 import inputs

TOL_R, TOL_A = 1e-13, 1e-100


def _rhs(A, w, c):
    return oracle.spmv(A, inputs.ones(A[0], w, c), w, c)


def test_real_standin_table1_shape():
    A = inputs.scaled_random_sparse()
    n, w = A[0], 2
    assert n == 765 and abs(len(A[2]) / n - 32) < 1e-9
    b = _rhs(A, w, 1)
    none = oracle.krylov("bicgstab", A, b, w, tol_rel=TOL_R, tol_abs=TOL_A, maxit=3 * n)
    assert none["status"] == "MAXIT" and none["iters"] == 3 * n
    for method in ("bicg", "cgs", "bicgstab", "gpbicg"):
        d = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=TOL_R, tol_abs=TOL_A, maxit=3 * n)
        p = oracle.krylov(method, A, b, w, ilu="mp", tol_rel=TOL_R, tol_abs=TOL_A, maxit=3 * n, mp_matrix=True)
        assert d["status"] == p["status"] == "OK"
        assert 3 <= d["iters"] <= 30 and abs(d["iters"] - p["iters"]) <= 1, (method, d["iters"], p["iters"])


def test_complex_standin_table2_shape():
    A = inputs.scaled_helmholtz2d()
    n, w, c = A[0], 2, 2
    assert n == 961
    n_, rp, ci, v = A
    D = np.zeros((n, n), complex)
    D[np.repeat(np.arange(n), np.diff(rp)), ci] = v[0::2] + 1j * v[1::2]
    assert np.array_equal(D, D.T)  # complex symmetric, not Hermitian
    b = _rhs(A, w, c)
    none = oracle.krylov("bicgstab", A, b, w, c, tol_rel=TOL_R, tol_abs=TOL_A, maxit=3 * n)
    assert none["status"] == "MAXIT" and none["iters"] == 3 * n
    d = oracle.krylov("bicg", A, b, w, c, ilu="fp64", tol_rel=TOL_R, tol_abs=TOL_A, maxit=3 * n)
    assert d["status"] == "OK" and 100 <= d["iters"] <= 3 * n
    assert d["relres_true"] < 1e-12
