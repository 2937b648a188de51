"""The paper-like "_p" build of the oracle (OpenMP SpMV, vector updates and inner products on all
host threads; the benchmark's all-core CPU baseline) computes what the plain oracle computes:
the SpMV row by row identically, inner products within the DD bound of the left-to-right sum,
and whole solves within the stated bars (tests/_bars.py)."""
import numpy as np
import pytest

import _bars
import oracle
from paper_2504_14498_gb300 import inputs

pytestmark = pytest.mark.skipif(oracle.lib_p() is None, reason="no OpenMP build of the oracle here")


def _with_p(fn):
    """Run fn with the "_p" library in place of the plain one (module-level functions use lib())."""
    saved = oracle._lib
    oracle._lib = oracle.lib_p()
    try:
        return fn()
    finally:
        oracle._lib = saved


def test_threads_reported():
    assert oracle.threads_p() >= 1


def test_spmv_identical():
    A = inputs.convdiff3d(13)[0]
    x = inputs.random_vector(A[0], 2, 1, seed=8)
    assert np.array_equal(_with_p(lambda: oracle.spmv(A, x, 2)), oracle.spmv(A, x, 2))


def test_dot_within_bound():
    oracle.threads_p(4)
    n = 50001
    a = inputs.random_vector(n, 2, 1, seed=1)
    b = inputs.random_vector(n, 2, 1, seed=2)
    got = _with_p(lambda: oracle.dot(a, b, n, 2))
    ref = oracle.dot(a, b, n, 2)
    mag = np.sum(np.abs(a[0::2] * b[0::2]))
    assert abs((got[0] - ref[0]) + (got[1] - ref[1])) <= 2.0 ** -100 * mag * 4


@pytest.mark.parametrize("ilu", ["fp64", "fp32"])
def test_solve_within_bars(ilu):
    A = inputs.convdiff2d(64, pe=10.0)
    n, w = A[0], 2
    b = oracle.spmv(A, inputs.ones(n, w), w)
    ref = oracle.krylov("bicgstab", A, b, w, ilu=ilu, tol_rel=1e-25, maxit=400)
    par = oracle.krylov("bicgstab", A, b, w, ilu=ilu, tol_rel=1e-25, maxit=400, parallel=True)
    assert par["status"] == ref["status"] == "OK"
    _bars.check_solve(par, ref, ilu, w, 1e-25)
    assert par["relres_true"] <= 1e-24
