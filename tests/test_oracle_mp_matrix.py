"""Pins of the oracle's SpMV with the matrix promoted to w components (the paper's rows without
"_d", Sec. 4) and of the Hermitian reading:
  * the promoted-matrix SpMV is within the format's bound of the exact product (rationals);
  * for D, TD and QD it equals the mixed SpMV bit for bit (every product and sum is exactly
    rounded in both), for DD it differs in rounding only;
  * Krylov runs with the promoted matrix and the multi-component factor (the plain rows
    "BiCG_ILU(0)" etc.) converge in the iterations of the "_d_ILU(0)" rows, to within one
    (Table 1);
  * for a Hermitian matrix the conjugate transpose used by BiCG is A itself.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2504_14498_gb300 import inputs
from _exact import F

BOUND = {1: Fraction(1, 2 ** 50), 2: Fraction(1, 2 ** 100), 3: Fraction(1, 2 ** 150), 4: Fraction(1, 2 ** 200)}


@pytest.mark.parametrize("c", [1, 2])
@pytest.mark.parametrize("w", [2, 3, 4])
def test_mp_matrix_spmv_exact_bound(w, c):
    A = inputs.random_sparse(40, 3, 9, seed=13, complex_=(c == 2))
    n, rp, ci, val = A
    x = inputs.random_vector(n, w, c, seed=3)
    y = oracle.spmv(A, x, w, c, mp_matrix=True).reshape(n, c, w)
    X = x.reshape(n, c, w)
    for i in range(n):
        er, ei, mag = Fraction(0), Fraction(0), Fraction(0)
        for p in range(rp[i], rp[i + 1]):
            j = int(ci[p])
            xr = F(X[j, 0])
            xi = F(X[j, 1]) if c == 2 else Fraction(0)
            ar = Fraction(float(val[c * p]))
            ai = Fraction(float(val[c * p + 1])) if c == 2 else Fraction(0)
            er += ar * xr - ai * xi
            ei += ar * xi + ai * xr
            mag += (abs(ar) + abs(ai)) * (abs(xr) + abs(xi))
        k = rp[i + 1] - rp[i]
        assert abs(F(y[i, 0]) - er) <= 4 * (k + 2) * BOUND[w] * mag
        if c == 2:
            assert abs(F(y[i, 1]) - ei) <= 4 * (k + 2) * BOUND[w] * mag


@pytest.mark.parametrize("c", [1, 2])
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_mp_matrix_spmv_vs_mixed(w, c):
    A = inputs.helmholtz2d(9, k=7.0) if c == 2 else inputs.convdiff2d(9, pe=10.0)
    x = inputs.random_vector(A[0], w, c, seed=5)
    mm = oracle.spmv(A, x, w, c, mp_matrix=True)
    mx = oracle.spmv(A, x, w, c)
    if w != 2:
        assert np.array_equal(mm, mx)
    else:
        assert not np.array_equal(mm, mx)  # DW*DW and DW*FP round differently ...
        lead = np.abs(mx.reshape(-1, c, w)[:, :, 0])
        assert np.all(np.abs((mm - mx).reshape(-1, c, w)[:, :, 0]) <= lead * 2.0 ** -100)  # ... by O(u^2)


@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
def test_plain_rows_match_d_rows_iterations(method):
    A = inputs.convdiff2d(20, pe=10.0)
    n, w = A[0], 2
    b = oracle.spmv(A, inputs.ones(n, w), w)
    plain = oracle.krylov(method, A, b, w, ilu="mp", tol_rel=1e-25, maxit=400, mp_matrix=True)
    d = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-25, maxit=400)
    assert plain["status"] == d["status"] == "OK"
    assert abs(plain["iters"] - d["iters"]) <= 1
    assert plain["relres_true"] < 1e-24


def test_hermitian_conjugate_transpose_is_A():
    A = inputs.magnetic_laplacian2d(7)
    n, rp, ci, val = A
    z = val[0::2] + 1j * val[1::2]
    D = np.zeros((n, n), complex)
    D[np.repeat(np.arange(n), np.diff(rp)), ci] = z
    assert np.array_equal(D, D.conj().T)
    # BiCG on a Hermitian system with an exactly Hermitian start (r~0 = r0) is CG-like: the
    # shadow residuals equal the residuals; it converges within n iterations in QD
    b = oracle.spmv(A, inputs.ones(n, 4, 2), 4, 2)
    out = oracle.krylov("bicg", A, b, 4, 2, tol_rel=1e-50, maxit=n)
    assert out["status"] == "OK" and out["iters"] <= n
