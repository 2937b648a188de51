"""Pins for the oracle's mixed SpMV, inner product, ILU(0) (Algorithm 1) and substitutions
(Algorithm 2).  References: exact rationals, library routines (sympy exact LU, scipy triangular
solves), and invariants of ILU(0):
  * SpMV / dot: |y_i - exact_i| <= tol * sum_j |a_ij||x_j| with tol = 2^-100 (DD), 2^-150 (TD),
    2^-200 (QD), k*2^-53 (D); the bound is row-relative because rows of conservative stencils can
    sum to exactly zero.
  * ILU(0): (L~U~)_ij = a_ij for every (i,j) in A's pattern (up to the rounding of the updates);
    ILU(0) equals the exact LU factorisation when no fill occurs (tridiagonal, full band).
  * Substitutions: M z = r and M^H z = r hold for the returned z; FP32 path is invariant under
    power-of-two scaling of r (the exponent rescale), including scales that underflow binary32.
"""
import random
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_2504_14498_gb300 import inputs
from tests._exact import F, U

TOL = {1: None, 2: Fraction(2) ** -100, 3: Fraction(2) ** -150, 4: Fraction(2) ** -200}


def _mat(A, c=1):
    n, rp, ci, val = A
    if c == 1:
        return sp.csr_matrix((val, ci, rp), shape=(n, n))
    v = val[0::2] + 1j * val[1::2]
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


@pytest.mark.parametrize("w", [1, 2, 3, 4])
@pytest.mark.parametrize("c", [1, 2])
def test_spmv_exact(w, c):
    A = inputs.random_sparse(40, 3, 12, seed=11 + w, complex_=(c == 2))
    n, rp, ci, val = A
    x = inputs.random_vector(n, w, c, seed=5 + w)
    y = oracle.spmv(A, x, w, c).reshape(n, c, w)
    X = x.reshape(n, c, w)
    for i in range(n):
        for part in range(c):
            ex = Fraction(0)
            mag = Fraction(0)
            k = rp[i + 1] - rp[i]
            for p in range(rp[i], rp[i + 1]):
                j = ci[p]
                if c == 1:
                    a = Fraction(val[p])
                    xv = F(X[j, 0])
                    ex += a * xv
                    mag += abs(a * xv)
                else:
                    ar, ai = Fraction(val[2 * p]), Fraction(val[2 * p + 1])
                    xr, xi = F(X[j, 0]), F(X[j, 1])
                    ex += (ar * xr - ai * xi) if part == 0 else (ar * xi + ai * xr)
                    mag += abs(ar * xr) + abs(ai * xi) if part == 0 else abs(ar * xi) + abs(ai * xr)
            tol = TOL[w] if w > 1 else (2 * k + 2) * U
            assert abs(F(y[i, part]) - ex) <= tol * mag, (i, part)


@pytest.mark.parametrize("w", [1, 2, 3, 4])
@pytest.mark.parametrize("c", [1, 2])
def test_dot_exact(w, c):
    n = 300
    a = inputs.random_vector(n, w, c, seed=21)
    b = inputs.random_vector(n, w, c, seed=22)
    got = oracle.dot(a, b, n, w, c)
    A, B = a.reshape(n, c, w), b.reshape(n, c, w)
    exr = exi = mag = Fraction(0)
    for i in range(n):
        if c == 1:
            t = F(A[i, 0]) * F(B[i, 0])
            exr += t
            mag += abs(t)
        else:
            ar, ai, br, bi = F(A[i, 0]), F(A[i, 1]), F(B[i, 0]), F(B[i, 1])
            exr += ar * br + ai * bi
            exi += ar * bi - ai * br
            mag += abs(ar * br) + abs(ai * bi) + abs(ar * bi) + abs(ai * br)
    tol = TOL[w] if w > 1 else 4 * n * U
    assert abs(F(got[:w]) - exr) <= tol * mag
    if c == 2:
        assert abs(F(got[w:]) - exi) <= tol * mag


def _dense_LU(A, fac, c=1):
    n, rp, ci, _ = A
    L = [[Fraction(0)] * n for _ in range(n)]
    Uu = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        L[i][i] = Fraction(1)
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            v = Fraction(fac[p]) if c == 1 else (Fraction(fac[2 * p]), Fraction(fac[2 * p + 1]))
            if j < i:
                L[i][j] = v
            else:
                Uu[i][j] = v
    return L, Uu


@pytest.mark.parametrize("prec,u", [("fp64", Fraction(1, 2 ** 53)), ("fp32", Fraction(1, 2 ** 24))])
@pytest.mark.parametrize("kind", ["convdiff", "random"])
def test_ilu0_pattern_invariant(prec, u, kind):
    """(L~ U~)_ij == a_ij on the pattern, within gamma_k * sum_k |l_ik||u_kj|."""
    if kind == "convdiff":
        A = inputs.convdiff2d(6, pe=3.0)
    else:
        A = inputs.random_sparse(30, 3, 8, seed=4)
    n, rp, ci, val = A
    st, fac, _ = oracle.ilu0(A, prec)
    assert st == 0
    L, Uu = _dense_LU(A, fac)
    a32 = val.astype(np.float32).astype(np.float64) if prec == "fp32" else val
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            s = Fraction(0)
            mag = Fraction(0)
            terms = 0
            for k in range(min(i, j) + 1):
                t = L[i][k] * Uu[k][j]
                if t != 0:
                    terms += 1
                s += t
                mag += abs(t)
            assert abs(s - Fraction(a32[p])) <= (terms + 2) * u * mag * Fraction(101, 100), (i, j)


def test_ilu0_has_fill_dropped():
    """On a 2-D 5-point matrix ILU(0) is not the exact LU: L~U~ differs from A off the pattern."""
    A = inputs.convdiff2d(5, pe=1.0)
    n, rp, ci, _ = A
    st, fac, _ = oracle.ilu0(A, "fp64")
    L, Uu = _dense_LU(A, fac)
    pat = {(i, ci[p]) for i in range(n) for p in range(rp[i], rp[i + 1])}
    off = max(abs(sum(L[i][k] * Uu[k][j] for k in range(n))) for i in range(n) for j in range(n) if (i, j) not in pat)
    assert off > 1e-3


@pytest.mark.parametrize("band", [1, 2])
def test_ilu0_equals_exact_lu_without_fill(band):
    """Tridiagonal (band 1) and full pentadiagonal band (band 2): ILU(0) = LU (sympy, exact)."""
    sympy = pytest.importorskip("sympy")
    n = 12
    rng = random.Random(band)
    rows, cols, vals = [], [], []
    dense = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        for j in range(max(0, i - band), min(n, i + band + 1)):
            v = Fraction(rng.randint(-8, 8), 8) if i != j else Fraction(rng.randint(40, 80), 8)
            dense[i][j] = v
            rows.append(i); cols.append(j); vals.append(float(v))
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    M.sort_indices()
    A = (n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    st, fac, _ = oracle.ilu0(A, "fp64")
    Ls, Us, perm = sympy.Matrix(dense).LUdecomposition()
    assert perm == []
    n_, rp, ci, _ = A
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            ex = Ls[i, j] if j < i else Us[i, j]
            ex = Fraction(int(ex.p), int(ex.q))
            if ex == 0:
                assert fac[p] == 0
            else:
                assert abs(Fraction(fac[p]) - ex) <= 8 * n * U * abs(ex)


def test_ilu0_bf16_is_rounded_fp32():
    A = inputs.convdiff2d(8, pe=5.0)
    _, f32, _ = oracle.ilu0(A, "fp32")
    _, b16, _ = oracle.ilu0(A, "bf16")
    bits = b16.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert np.all(np.abs(b16 - f32) <= np.abs(f32) * 2.0 ** -8)


def test_ilu0_complex_invariant():
    A = inputs.helmholtz2d(5, k=3.0)
    n, rp, ci, val = A
    st, fac, _ = oracle.ilu0(A, "fp64", c=2)
    assert st == 0
    Lc = np.eye(n, dtype=complex)
    Uc = np.zeros((n, n), dtype=complex)
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            v = fac[2 * p] + 1j * fac[2 * p + 1]
            if j < i:
                Lc[i, j] = v
            else:
                Uc[i, j] = v
    P = Lc @ Uc
    Ad = _mat(A, 2).toarray()
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            assert abs(P[i, j] - Ad[i, j]) <= 1e-14 * (abs(Ad[i, j]) + 1)


def test_ilu0_errors():
    # zero pivot at row 1: a11 - a10 a01 / a00 = 1 - 1*1/1 = 0
    A = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 1.0, 1.0, 1.0]))
    st, _, fr = oracle.ilu0(A)
    assert oracle.STATUS[st] == "ZERO_PIVOT" and fr == 1
    B = (2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    st, _, fr = oracle.ilu0(B)
    assert oracle.STATUS[st] == "MISSING_DIAG" and fr == 0
    C = (2, np.array([0, 2, 3], np.int32), np.array([1, 0, 1], np.int32), np.array([1.0, 2.0, 3.0]))
    st, _, fr = oracle.ilu0(C)
    assert oracle.STATUS[st] == "INVALID_ARG" and fr == 0


def _factor_mats(A, fac, c):
    n, rp, ci, _ = A
    Lm = np.eye(n, dtype=complex if c == 2 else float)
    Um = np.zeros((n, n), dtype=complex if c == 2 else float)
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            v = fac[p] if c == 1 else fac[2 * p] + 1j * fac[2 * p + 1]
            if j < i:
                Lm[i, j] = v
            else:
                Um[i, j] = v
    return Lm, Um


@pytest.mark.parametrize("c", [1, 2])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_substitution_solves_M(c, trans, prec):
    A = inputs.random_sparse(60, 3, 9, seed=9, complex_=(c == 2))
    n = A[0]
    st, fac, _ = oracle.ilu0(A, prec, c)
    assert st == 0
    w = 2
    r = inputs.random_vector(n, w, c, seed=31)
    z = oracle.precond(A, fac, r, w, prec, c, trans).reshape(n, c, w)
    Lm, Um = _factor_mats(A, fac, c)
    M = Lm @ Um
    if trans:
        M = M.conj().T
    zz = z[:, 0, 0] + (1j * z[:, 1, 0] if c == 2 else 0)
    rr = r.reshape(n, c, w)[:, 0, 0] + (1j * r.reshape(n, c, w)[:, 1, 0] if c == 2 else 0)
    res = np.linalg.norm(M @ zz - rr) / np.linalg.norm(rr)
    assert res < (1e-14 if prec == "fp64" else 1e-5)


def test_substitution_matches_scipy_triangular():
    A = inputs.convdiff2d(10, pe=4.0)
    n = A[0]
    st, fac, _ = oracle.ilu0(A, "fp64")
    r = inputs.random_vector(n, 1, 1, seed=2)
    z = oracle.precond(A, fac, r, 1, "fp64")
    Lm, Um = _factor_mats(A, fac, 1)
    y = spla.spsolve_triangular(sp.csr_matrix(Lm), r, lower=True, unit_diagonal=True)
    zs = spla.spsolve_triangular(sp.csr_matrix(Um), y, lower=False)
    assert np.max(np.abs(z - zs)) <= 1e-12 * np.max(np.abs(zs))


def test_substitution_dd_exact_rational():
    """The DD (paper's _d) solve against the exact rational solution of L~U~ z = r."""
    A = inputs.random_sparse(12, 2, 5, seed=13)
    n, rp, ci, _ = A
    st, fac, _ = oracle.ilu0(A, "fp64")
    w = 4
    r = inputs.random_vector(n, w, 1, seed=3)
    z = oracle.precond(A, fac, r, w, "fp64").reshape(n, w)
    L, Uu = _dense_LU(A, fac)
    R = [F(r.reshape(n, w)[i]) for i in range(n)]
    y = [Fraction(0)] * n
    for i in range(n):
        y[i] = R[i] - sum(L[i][j] * y[j] for j in range(i))
    zx = [Fraction(0)] * n
    for i in reversed(range(n)):
        zx[i] = (y[i] - sum(Uu[i][j] * zx[j] for j in range(i + 1, n))) / Uu[i][i]
    scale = max(abs(v) for v in zx)
    for i in range(n):
        assert abs(F(z[i]) - zx[i]) <= Fraction(2) ** -190 * scale


@pytest.mark.parametrize("shift", [-600, -300, 0, 300])
def test_fp32_path_power_of_two_invariance(shift):
    """The binary32 path rescales by 2^-e before rounding: results scale exactly with r,
    even where r itself would underflow or overflow binary32."""
    A = inputs.convdiff2d(8, pe=2.0)
    n = A[0]
    st, fac, _ = oracle.ilu0(A, "fp32")
    r = inputs.random_vector(n, 2, 1, seed=8)
    z0 = oracle.precond(A, fac, r, 2, "fp32")
    z1 = oracle.precond(A, fac, np.ldexp(r, shift), 2, "fp32")
    assert np.array_equal(np.ldexp(z0, shift), z1)
    assert np.any(z1 != 0)


@pytest.mark.parametrize("prec,u", [("fp64", Fraction(1, 2 ** 53)), ("fp32", Fraction(1, 2 ** 24))])
def test_ilu0_complex_pattern_invariant(prec, u):
    """(L~ U~)_ij == a_ij on the pattern for a complex matrix whose off-diagonal entries are
    complex too (every update l_ik u_kj has four nonzero real products; on a mesh with real
    couplings the imaginary parts of u_kj stay 0 and the cross terms are never exercised), within
    (terms + 4) * 4u * sum_k |l_ik| |u_kj| per component."""
    A = inputs.random_sparse(40, 3, 9, seed=21, complex_=True, weak_frac=0.0)
    n, rp, ci, val = A
    st, fac, _ = oracle.ilu0(A, prec, c=2)
    assert st == 0
    L, Uu = _dense_LU(A, fac, c=2)
    one = (Fraction(1), Fraction(0))
    for i in range(n):
        L[i][i] = one
    src = val.astype(np.float32).astype(np.float64) if prec == "fp32" else val
    updates = 0
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            sr = si = Fraction(0)
            mag = Fraction(0)
            terms = 0
            for k in range(min(i, j) + 1):
                lk, uk = L[i][k], Uu[k][j]
                if not isinstance(lk, tuple) or not isinstance(uk, tuple):
                    continue
                tr = lk[0] * uk[0] - lk[1] * uk[1]
                ti = lk[0] * uk[1] + lk[1] * uk[0]
                if tr != 0 or ti != 0:
                    terms += 1
                    if k != min(i, j) and lk[1] != 0 and uk[1] != 0:
                        updates += 1
                sr += tr
                si += ti
                mag += (abs(lk[0]) + abs(lk[1])) * (abs(uk[0]) + abs(uk[1]))
            bound = (terms + 4) * 4 * u * mag
            assert abs(sr - Fraction(src[2 * p])) <= bound, (i, j, "re")
            assert abs(si - Fraction(src[2 * p + 1])) <= bound, (i, j, "im")
    assert updates > 0  # the cross terms of complex updates were exercised
