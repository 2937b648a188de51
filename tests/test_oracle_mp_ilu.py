"""Pins of the oracle's ILU(0) in the working multi-component precision (the paper's rows
without "_d"), against exact rational arithmetic (Python Fraction):
  * the factor reproduces A on its pattern to within the multi-component rounding;
  * without fill (tridiagonal, banded) the factor is the exact LU rounded to w components;
  * the substitutions solve M z = r and M^H z = r with the multi-component factor.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2504_14498_gb300 import inputs
from _exact import F

TOLW = {2: Fraction(1, 2 ** 100), 4: Fraction(1, 2 ** 195)}


def _entries(A, fac, w, c):
    """Exact values of the factor entries (complex: pairs)."""
    n, rp, ci, _ = A
    f = fac.reshape(-1, c, w)
    return [tuple(F(f[p, k]) for k in range(c)) for p in range(len(ci))]


def _lu_products(A, E, c):
    """(L~U~)_ij on A's pattern and sum |L~_ik||U~_kj| (bounds), exactly; real (c = 1) only."""
    n, rp, ci, _ = A
    pos = {}
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            pos[(i, int(ci[p]))] = p
    out = {}
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = int(ci[p])
            s, mag = Fraction(0), Fraction(0)
            for k in range(min(i, j) + 1):
                lik = Fraction(1) if k == i else (E[pos[(i, k)]][0] if (i, k) in pos and k < i else None)
                ukj = E[pos[(k, j)]][0] if (k, j) in pos and k <= j else None
                if lik is None or ukj is None:
                    continue
                s += lik * ukj
                mag += abs(lik) * abs(ukj)
            out[(i, j)] = (s, mag)
    return out


@pytest.mark.parametrize("w", [2, 4])
def test_mp_factor_reproduces_A_on_pattern(w):
    A = inputs.random_sparse(14, 3, 6, seed=31)
    st, fac, _ = oracle.ilu0(A, "mp", 1, w)
    assert st == 0
    E = _entries(A, fac, w, 1)
    prods = _lu_products(A, E, 1)
    n, rp, ci, val = A
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            s, mag = prods[(i, int(ci[p]))]
            assert abs(s - Fraction(float(val[p]))) <= 8 * TOLW[w] * mag


@pytest.mark.parametrize("w", [2, 4])
def test_mp_factor_is_rounded_exact_lu_without_fill(w):
    n = 10
    T = inputs.tridiag(n, -1.3, 4.1, -0.7)
    st, fac, _ = oracle.ilu0(T, "mp", 1, w)
    assert st == 0
    E = _entries(T, fac, w, 1)
    # exact LU of the tridiagonal matrix in rationals
    lo, di, up = Fraction(-1.3), Fraction(4.1), Fraction(-0.7)
    u_prev = None
    p = 0
    _, rp, ci, _ = T
    for i in range(n):
        u_ii = di if i == 0 else di - (lo / u_prev) * up
        for q in range(rp[i], rp[i + 1]):
            j = int(ci[q])
            exact = lo / u_prev if j == i - 1 else (u_ii if j == i else up)
            assert abs(E[q][0] - exact) <= 4 * TOLW[w] * abs(exact), (i, j)
        u_prev = u_ii


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("c", [1, 2])
def test_mp_substitutions_solve_M(c, trans):
    w = 2
    A = inputs.random_sparse(12, 3, 5, seed=41, complex_=(c == 2))
    n, rp, ci, _ = A
    st, fac, _ = oracle.ilu0(A, "mp", c, w)
    assert st == 0
    r = inputs.random_vector(n, w, c, seed=5)
    z = oracle.precond(A, fac, r, w, "mp", c, trans)
    # exact residual of M z = r (or M^H z = r) with M = L~ U~ from the factor entries
    f = fac.reshape(-1, c, w)
    Lm = [[Fraction(0)] * n for _ in range(n)]
    Um = [[Fraction(0)] * n for _ in range(n)]
    Li = [[Fraction(0)] * n for _ in range(n)]
    Ui = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        Lm[i][i] = Fraction(1)
        for p in range(rp[i], rp[i + 1]):
            j = int(ci[p])
            re = F(f[p, 0])
            im = F(f[p, 1]) if c == 2 else Fraction(0)
            if j < i:
                Lm[i][j], Li[i][j] = re, im
            else:
                Um[i][j], Ui[i][j] = re, im
    zz = z.reshape(n, c, w)
    rr = r.reshape(n, c, w)
    zr = [F(zz[i, 0]) for i in range(n)]
    zi = [F(zz[i, 1]) if c == 2 else Fraction(0) for i in range(n)]

    def mat(Xr, Xi, vr, vi, conj_t):
        out_r, out_i = [], []
        for i in range(n):
            sr, si = Fraction(0), Fraction(0)
            for j in range(n):
                ar, ai = (Xr[j][i], -Xi[j][i]) if conj_t else (Xr[i][j], Xi[i][j])
                sr += ar * vr[j] - ai * vi[j]
                si += ar * vi[j] + ai * vr[j]
            out_r.append(sr)
            out_i.append(si)
        return out_r, out_i

    if not trans:  # L (U z)
        yr, yi = mat(Um, Ui, zr, zi, False)
        mr, mi = mat(Lm, Li, yr, yi, False)
    else:  # U^H (L^H z)
        yr, yi = mat(Lm, Li, zr, zi, True)
        mr, mi = mat(Um, Ui, yr, yi, True)
    scale = max(abs(F(rr[i, k])) for i in range(n) for k in range(c))
    for i in range(n):
        assert abs(mr[i] - F(rr[i, 0])) <= Fraction(1, 2 ** 90) * scale * 100
        if c == 2:
            assert abs(mi[i] - F(rr[i, 1])) <= Fraction(1, 2 ** 90) * scale * 100


def test_mp_factor_krylov_matches_paper_observation():
    """Table 1: the binary64-substitution rows ("_d_ILU(0)") need the same iteration counts as the
    multi-component ILU(0) rows, to within one; the oracle's two factors behave the same way."""
    A = inputs.convdiff2d(20, pe=10.0)
    n = A[0]
    for w, tol in ((2, 1e-25), (4, 1e-55)):
        b = oracle.spmv(A, inputs.ones(n, w), w)
        mp = oracle.krylov("bicgstab", A, b, w, ilu="mp", tol_rel=tol, maxit=300)
        d = oracle.krylov("bicgstab", A, b, w, ilu="fp64", tol_rel=tol, maxit=300)
        assert mp["status"] == d["status"] == "OK"
        assert abs(mp["iters"] - d["iters"]) <= 1
