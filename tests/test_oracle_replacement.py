"""Pins for the oracle's residual replacement (the periodic true residual b - A x; the paper
recomputes nothing, the rule is this project's reading): with a period P > 0 the true residual is
formed at every multiple of P and whenever the recursive norm passes the stopping test; above
10x the target it replaces r, and a passed test is withdrawn.

Pinned against quantities the oracle does not compute itself:
  * exact rational residuals ||b - A x||^2 of the returned iterate (Python Fractions): the
    unpreconditioned DD runs on a Peclet-10 convection-diffusion matrix stop on a recursive
    residual far below their true one without the rule (CGS: true residual ~1e-6 for a target of
    1e-25), and end within 10x the target with it;
  * the check schedule (multiples of P and the iterations whose recursive norm passed the test);
  * the last recorded true norm against the exact norm of the returned iterate;
  * a run whose test stands at the first check is the run without the rule, bit for bit.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2504_14498_gb300 import inputs

METHODS = ["bicg", "cgs", "bicgstab", "gpbicg"]


def _exact_res2(A, b, x, w):
    """||b - A x||_2^2 in exact rationals (real A, w-component b and x)."""
    n, rp, ci, val = A
    X = [sum((Fraction(float(c)) for c in x[i * w:(i + 1) * w]), Fraction(0)) for i in range(n)]
    tot = Fraction(0)
    for i in range(n):
        s = sum((Fraction(float(c)) for c in b[i * w:(i + 1) * w]), Fraction(0))
        for p in range(rp[i], rp[i + 1]):
            s -= Fraction(float(val[p])) * X[ci[p]]
        tot += s * s
    return tot


@pytest.fixture(scope="module")
def drift_case():
    A = inputs.convdiff2d(33, pe=10.0)
    n, w = A[0], 2
    b = oracle.spmv(A, inputs.ones(n, w), w)
    return A, b, w


def test_false_convergence_without_the_rule(drift_case):
    A, b, w = drift_case
    out = oracle.krylov("cgs", A, b, w, ilu="none", tol_rel=1e-25, maxit=3000, true_res_period=0)
    assert out["status"] == "OK" and out["replacements"] == 0
    r0 = out["hist"][0]
    assert out["hist"][-1] < 1e-25 * r0                       # the recursive test passed ...
    assert _exact_res2(A, b, out["x"], w) > Fraction(1e-12 * r0) ** 2  # ... far from the truth


@pytest.mark.parametrize("method", METHODS)
def test_rule_restores_the_true_residual(drift_case, method):
    A, b, w = drift_case
    tol = 1e-25
    out = oracle.krylov(method, A, b, w, ilu="none", tol_rel=tol, maxit=3000, true_res_period=50)
    assert out["status"] == "OK"
    assert out["replacements"] >= 1
    r0 = out["hist"][0]
    exact = _exact_res2(A, b, out["x"], w)
    assert exact <= (Fraction(10 * tol * r0) * (1 + Fraction(1, 10 ** 6))) ** 2
    # the last recorded true norm is the norm of the returned iterate's residual
    last = out["hist_true"][out["iters"]]
    assert abs(last ** 2 - float(exact)) <= 1e-4 * float(exact)


@pytest.mark.parametrize("method", METHODS)
def test_check_schedule(drift_case, method):
    A, b, w = drift_case
    tol, P = 1e-25, 7
    out = oracle.krylov(method, A, b, w, ilu="none", tol_rel=tol, maxit=3000, true_res_period=P)
    h, ht = out["hist"], out["hist_true"]
    thr = tol * h[0]
    for k in range(1, out["iters"] + 1):
        checked = (k % P == 0) or (h[k] < thr)
        assert (not np.isnan(ht[k])) == checked, k
        if checked and k < out["iters"]:
            # a check that did not end the run found the true norm above 10x the target
            # (replacement) or was a periodic check whose true norm was below it
            assert ht[k] > 10 * thr or k % P == 0
    # the run ended on a check that accepted
    assert ht[out["iters"]] <= 10 * thr and h[out["iters"]] < thr


@pytest.mark.parametrize("method", METHODS)
def test_standing_test_is_the_plain_run(method):
    A = inputs.convdiff2d(33, pe=10.0)
    n, w = A[0], 2
    b = oracle.spmv(A, inputs.ones(n, w), w)
    plain = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-25, maxit=600, true_res_period=0)
    ruled = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-25, maxit=600, true_res_period=500)
    assert plain["status"] == ruled["status"] == "OK"
    assert ruled["replacements"] == 0
    assert np.array_equal(plain["hist"], ruled["hist"])
    assert np.array_equal(plain["x"], ruled["x"])
    k = ruled["iters"]
    assert np.sum(~np.isnan(ruled["hist_true"])) == 1 and ruled["hist_true"][k] <= 10 * 1e-25 * ruled["hist"][0]
    assert ruled["hist_true"][k] == pytest.approx(ruled["relres_true"] * ruled["hist"][0], rel=1e-12)


def test_threshold_is_ten_times_the_target(drift_case):
    """At a passed test the decision follows the 10x threshold: here the first passed test meets
    a true norm between 10x and 1000x the target, so it is withdrawn and r replaced."""
    A, b, w = drift_case
    tol = 1e-24
    out = oracle.krylov("bicgstab", A, b, w, ilu="none", tol_rel=tol, maxit=3000, true_res_period=10 ** 6)
    h, ht = out["hist"], out["hist_true"]
    thr = tol * h[0]
    k1 = next(k for k in range(1, len(h)) if h[k] < thr)
    assert 10 * thr < ht[k1] < 1000 * thr  # the case sits where the threshold decides
    assert out["iters"] > k1 and out["replacements"] >= 1
    assert out["status"] == "OK" and ht[out["iters"]] <= 10 * thr
