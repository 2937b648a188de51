"""Pins for the oracle's Krylov solvers (Algorithm 3 BiCG; CGS, BiCGSTAB, GPBiCG as read in
Sec. 3) against mathematics that does not depend on the oracle:
  * finite termination: on tiny nonsymmetric systems every method reaches the solution within n
    iterations (Krylov dimension), checked in QD where rounding is far below the test;
  * manufactured solutions b = A x* (x* = ones, and the paper's x = sqrt(2)[1..n] of Sec. 4);
  * reductions: GPBiCG with eta forced to 0 follows BiCGSTAB; BiCG without preconditioner on a
    symmetric positive definite matrix follows conjugate gradients (scipy's cg);
  * M = A (ILU(0) exact, exactly representable factors): convergence in one iteration;
  * statuses: breakdown, NaN in b, maximum iterations; with / without ILU(0) (the qualitative
    observation of Sec. 4 that the unpreconditioned methods need far more iterations).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_2504_14498_gb300 import inputs

METHODS = ["bicg", "cgs", "bicgstab", "gpbicg"]


def _rhs(A, x, w, c=1):
    return oracle.spmv(A, x, w, c)


def _hi(v, n, w, c=1):
    v = v.reshape(n, c, w)
    return v[:, 0, 0] + (1j * v[:, 1, 0] if c == 2 else 0)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("c", [1, 2])
def test_finite_termination(method, c):
    n = 7
    A = inputs.random_sparse(n, 3, 6, seed=100 + c, complex_=(c == 2), weak_frac=0.0)
    w = 4
    xs = inputs.random_vector(n, w, c, seed=4)
    b = _rhs(A, xs, w, c)
    out = oracle.krylov(method, A, b, w, c, ilu="none", tol_rel=1e-45, maxit=n)
    assert out["status"] == "OK", out["status"]
    assert out["iters"] <= n
    err = np.max(np.abs(_hi(out["x"], n, w, c) - _hi(xs, n, w, c)))
    assert err < 1e-40


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("ilu", ["fp64", "fp32", "bf16"])
def test_manufactured_convdiff_dd(method, ilu):
    m = 12
    A = inputs.convdiff2d(m, pe=10.0)
    n = A[0]
    w = 2
    xs = inputs.ones(n, w)
    b = _rhs(A, xs, w)
    out = oracle.krylov(method, A, b, w, ilu=ilu, tol_rel=1e-25, maxit=400)
    assert out["status"] == "OK"
    assert out["relres_true"] < 1e-24
    assert np.max(np.abs(out["x"].reshape(n, w)[:, 0] - 1.0)) < 1e-20
    # recursive residual history is what the stopping rule saw
    assert out["hist"][-1] < 1e-25 * out["hist"][0]


@pytest.mark.parametrize("method", METHODS)
def test_manufactured_paper_xstar_complex_qd(method):
    """Sec. 4 exact solution for complex systems, x = sqrt(2+3i) [1..n], QD vectors."""
    A = inputs.helmholtz2d(6, k=4.0)
    n, w, c = A[0], 4, 2
    xs = inputs.paper_xstar(n, w, complex_=True)
    b = _rhs(A, xs, w, c)
    out = oracle.krylov(method, A, b, w, c, ilu="fp64", tol_rel=1e-55, maxit=300)
    assert out["status"] == "OK"
    rel = np.max(np.abs(_hi(out["x"], n, w, c) - _hi(xs, n, w, c))) / np.max(np.abs(_hi(xs, n, w, c)))
    assert rel < 1e-15  # leading components agree to binary64 rounding
    assert out["relres_true"] < 1e-54


def test_gpbicg_eta0_is_bicgstab():
    A = inputs.convdiff2d(10, pe=5.0)
    n, w = A[0], 2
    b = _rhs(A, inputs.ones(n, w), w)
    g = oracle.krylov("gpbicg", A, b, w, ilu="fp64", tol_rel=1e-25, maxit=300, force_eta0=True)
    s = oracle.krylov("bicgstab", A, b, w, ilu="fp64", tol_rel=1e-25, maxit=300)
    k = min(len(g["hist"]), len(s["hist"]), 12)
    np.testing.assert_allclose(g["hist"][:k], s["hist"][:k], rtol=1e-12)
    assert abs(g["iters"] - s["iters"]) <= 1
    # without the forcing, GPBiCG is a different method
    full = oracle.krylov("gpbicg", A, b, w, ilu="fp64", tol_rel=1e-25, maxit=300)
    assert not np.allclose(full["hist"][2:k], s["hist"][2:k], rtol=1e-6)


def test_bicg_is_cg_on_spd():
    m = 10
    A = inputs.convdiff2d(m, pe=0.0)  # pure diffusion: symmetric positive definite
    n, rp, ci, val = A
    S = sp.csr_matrix((val, ci, rp), shape=(n, n))
    bb = np.sin(np.arange(n) + 1.0)
    res = []
    spla.cg(S, bb, rtol=1e-30, maxiter=12, callback=lambda xk: res.append(np.linalg.norm(bb - S @ xk)))
    out = oracle.krylov("bicg", A, bb.copy(), 1, ilu="none", tol_rel=1e-30, maxit=12)
    k = min(len(res), 10)
    np.testing.assert_allclose(out["hist"][1:k + 1], res[:k], rtol=1e-8)


def _exact_lu_tridiag(n):
    """A = L U with L unit lower bidiagonal (sub-diagonal 1/2) and U upper bidiagonal (diagonal 4,
    super-diagonal -1): all entries of A and of its ILU(0) = LU factors are exact binary64."""
    lo = np.full(n, 0.5 * 4.0)  # l_{i,i-1} u_{i-1,i-1} = 0.5 * 4
    di = np.full(n, 4.0)
    di[1:] = 4.0 + 0.5 * -1.0   # l u_{i-1,i} + u_ii
    up = np.full(n, -1.0)
    return inputs.tridiag(n, lo, di, up)


@pytest.mark.parametrize("method", METHODS)
def test_one_iteration_when_M_equals_A(method):
    n = 50
    A = _exact_lu_tridiag(n)
    st, fac, _ = oracle.ilu0(A, "fp64")
    assert st == 0
    rp, ci = A[1], A[2]
    for i in range(n):  # factors are exactly L (0.5) and U (4, -1)
        for p in range(rp[i], rp[i + 1]):
            expect = 0.5 if ci[p] < i else (4.0 if ci[p] == i else -1.0)
            assert fac[p] == expect
    w = 2
    b = _rhs(A, inputs.paper_xstar(n, w), w)
    out = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-28, maxit=5)
    assert out["status"] == "OK" and out["iters"] == 1


def test_breakdown_status():
    # A = [[0,1],[1,0]], b = e1: <r~, A r> = 0 at the first step
    A = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([0.0, 1.0, 1.0, 0.0]))
    b = np.array([1.0, 0.0, 0.0, 0.0])
    for m in METHODS:
        out = oracle.krylov(m, A, b, 2, ilu="none", maxit=10)
        assert out["status"] == "BREAKDOWN", m


@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_bicgstab_omega_zero_is_breakdown(w):
    """omega = <t, s> / <t, t> = 0 makes the next beta = (rho_new / rho)(alpha / omega) divide
    by zero, so it is a breakdown.  A = [[0, -1], [1, 0]] (skew), b = e1, shadow (1, 49): alpha =
    1/49 rounded, s = (1, -alpha), t = A s = (alpha, 1), and <t, s> = alpha - alpha = 0 exactly,
    while rho_new = <r~, s> = 1 - 49 alpha is not 0 after rounding in D, TD and QD (in exact
    arithmetic it would be, and the rho test would catch it; in DD the product rounds back to 1
    and the rho test fires on the same iteration).  Expected: BREAKDOWN after 1 iteration,
    x = alpha b."""
    A = (2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([-1.0, 1.0]))
    b = np.zeros(2 * w)
    b[0] = 1.0
    shadow = np.zeros(2 * w)
    shadow[0], shadow[w] = 1.0, 49.0
    out = oracle.krylov("bicgstab", A, b, w, shadow=shadow, maxit=10)
    assert out["status"] == "BREAKDOWN" and out["iters"] == 1
    alpha = oracle.mp_op("div", w, [1.0] + [0.0] * (w - 1), [49.0] + [0.0] * (w - 1))
    assert np.array_equal(out["x"][:w], alpha) and not np.any(out["x"][w:])


def test_gpbicg_zeta_zero_is_breakdown():
    """GPBiCG's first step is BiCGSTAB's (eta = 0, zeta = <c, t> / <c, c>), so on the skew system
    above zeta is exactly 0; the next beta = (alpha / zeta)(...) would divide by it: BREAKDOWN
    after 1 iteration in every format where the rho test does not fire first."""
    A = (2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([-1.0, 1.0]))
    for w in (1, 3, 4):
        b = np.zeros(2 * w)
        b[0] = 1.0
        shadow = np.zeros(2 * w)
        shadow[0], shadow[w] = 1.0, 49.0
        out = oracle.krylov("gpbicg", A, b, w, shadow=shadow, maxit=10)
        assert out["status"] == "BREAKDOWN" and out["iters"] == 1, w


@pytest.mark.parametrize("w", [1, 2, 4])
def test_gpbicg_singular_least_squares_is_breakdown(w):
    """GPBiCG's two-term minimisation ||t - eta y - zeta c|| has a singular 2x2 system when y and c
    are parallel (det = <c,c><y,y> - <c,y><y,c> = 0).  On this 3x3 integer system with a shadow
    residual every scalar of the first two steps is a dyadic rational, so each format computes
    them exactly (alpha = 1/4, zeta = 1/4, beta = -3/8, then alpha = -2), and at the second step
    c = (0, 0, -9) and y = (0, 0, -9/2) = c/2 (found by an exact rational search): BREAKDOWN after
    1 completed iteration."""
    D = [[2, 1, 0], [2, 0, 0], [-2, -2, 2]]
    rp, ci, v = [0], [], []
    for row in D:
        for j, a in enumerate(row):
            if a:
                ci.append(j)
                v.append(float(a))
        rp.append(len(ci))
    A = (3, np.array(rp, np.int32), np.array(ci, np.int32), np.array(v))
    b = np.zeros(3 * w)
    b[::w] = [-2.0, 0.0, -1.0]
    shadow = np.zeros(3 * w)
    shadow[::w] = [-1.0, -1.0, 0.0]
    out = oracle.krylov("gpbicg", A, b, w, shadow=shadow, maxit=10)
    assert out["status"] == "BREAKDOWN" and out["iters"] == 1


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("w", [1, 2])
def test_breakdown_rho_zero(method, w):
    """rho = <r~, r> = 0 with r != 0 (a shadow residual orthogonal to r0) is a breakdown before
    the first step: BREAKDOWN after 0 iterations and x = x0 (otherwise alpha = 0 and the
    iteration would stall until maxit)."""
    A = inputs.convdiff2d(4, pe=3.0)
    n = A[0]
    b = _rhs(A, inputs.ones(n, w), w)
    bh = b.reshape(n, w)[:, 0]
    assert not np.any(b.reshape(n, w)[:, 1:])  # integer row sums: exact leading parts
    shadow = np.zeros(n * w)
    shadow[0], shadow[w] = bh[1], -bh[0]
    out = oracle.krylov(method, A, b, w, shadow=shadow, maxit=20)
    assert out["status"] == "BREAKDOWN" and out["iters"] == 0
    assert not np.any(out["x"])


def test_nan_and_maxit():
    A = inputs.convdiff2d(8, pe=10.0)
    n, w = A[0], 2
    b = _rhs(A, inputs.ones(n, w), w)
    bn = b.copy()
    bn[5 * w] = np.nan
    assert oracle.krylov("bicgstab", A, bn, w, ilu="fp64")["status"] == "NAN"
    out = oracle.krylov("bicgstab", A, b, w, ilu="none", maxit=3)
    assert out["status"] == "MAXIT" and out["iters"] == 3


@pytest.mark.parametrize("method", METHODS)
def test_stopping_rule_both_terms(method):
    """Algorithm 3's test ||r_k|| < eps_r ||r_0|| + eps_a, both terms: with eps_r = 0 the run stops
    at the first k whose recorded norm is below eps_a (and not before), with eps_a = 0 at the
    first below eps_r ||r_0||; a larger eps_a stops earlier."""
    A = inputs.convdiff2d(10, pe=10.0)
    n, w = A[0], 2
    b = _rhs(A, inputs.ones(n, w), w)
    ref = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-28, maxit=200)
    r0 = ref["hist"][0]
    for tol_rel, tol_abs in ((0.0, 1e-6 * r0), (1e-6, 0.0), (1e-9, 1e-6 * r0)):
        out = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=tol_rel, tol_abs=tol_abs, maxit=200)
        tol = tol_rel * r0 + tol_abs
        h = out["hist"]
        assert out["status"] == "OK"
        assert h[-1] < tol and np.all(h[:-1] >= tol), (tol_rel, tol_abs, h)
        assert np.array_equal(h, ref["hist"][: len(h)])  # the same iterates until it stops
    early = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-12, tol_abs=1e-3 * r0, maxit=200)
    assert early["iters"] < oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-12, maxit=200)["iters"]


def test_ilu_needed_paper_setting():
    """Sec. 4 setting (eps_r = 1e-13, eps_a = 1e-100, maxit = 3n) on the config-1 stand-in:
    with ILU(0) each method converges, and needs far fewer iterations than without it."""
    A = inputs.convdiff2d(24, pe=10.0)
    n, w = A[0], 2
    b = _rhs(A, inputs.paper_xstar(n, w), w)
    for m in METHODS:
        pre = oracle.krylov(m, A, b, w, ilu="fp64", tol_rel=1e-13, tol_abs=1e-100, maxit=3 * n)
        non = oracle.krylov(m, A, b, w, ilu="none", tol_rel=1e-13, tol_abs=1e-100, maxit=3 * n)
        assert pre["status"] == "OK"
        assert 3 * pre["iters"] < non["iters"], (m, pre["iters"], non["iters"])


@pytest.mark.parametrize("method", ["cgs", "bicgstab", "gpbicg"])
def test_hat_form_equals_definitional_form(method):
    """The right-preconditioned forms run on A with M^-1 applied inside (the "hat" vectors) equal
    the unpreconditioned method on the explicit operator A~ = A M^-1 (dense, each entry rounded to
    binary64 once), residual norm for residual norm: r = b - A x = b - A~ y with x = M^-1 y.  A
    mis-stated recurrence in any of these forms separates the two histories immediately.  (BiCG
    of Algorithm 3 is the two-sided form, M z = r and M^H z~ = r~: it equals BiCG on A~ started
    from the shadow M^-H r0 instead of r0, so it is pinned by the M = A and CG reductions.)"""
    n, w = 8, 4
    A = inputs.random_sparse(n, 3, 5, seed=61, weak_frac=0.0)
    _, rp, ci, val = A
    st, fac, _ = oracle.ilu0(A, "fp64")
    assert st == 0
    F = np.zeros((n, n))
    F[np.repeat(np.arange(n), np.diff(rp)), ci] = fac
    Mm = (np.tril(F, -1) + np.eye(n)) @ np.triu(F)
    D = np.zeros((n, n))
    D[np.repeat(np.arange(n), np.diff(rp)), ci] = val
    At = D @ np.linalg.inv(Mm)
    At_csr = (n, np.arange(0, n * n + 1, n, dtype=np.int32), np.tile(np.arange(n, dtype=np.int32), n), At.reshape(-1))
    b = inputs.random_vector(n, w, 1, seed=8)
    hat = oracle.krylov(method, A, b, w, ilu="fp64", tol_rel=1e-40, maxit=n)
    defn = oracle.krylov(method, At_csr, b, w, ilu="none", tol_rel=1e-40, maxit=n)
    k = min(len(hat["hist"]), len(defn["hist"]), 5)
    assert k >= 4
    np.testing.assert_allclose(hat["hist"][:k], defn["hist"][:k], rtol=1e-9)


def test_bicg_two_sided_equals_bicg_on_explicit_operator():
    """Algorithm 3 (M z = r, M^H z~ = r~) equals unpreconditioned BiCG on A~ = A M^-1 started from
    the shadow M^-H r0, residual for residual (the derivation: z~ = M^-H r~ carries the shadow of
    the explicit form)."""
    n, w = 8, 4
    A = inputs.random_sparse(n, 3, 5, seed=63, weak_frac=0.0)
    _, rp, ci, val = A
    st, fac, _ = oracle.ilu0(A, "fp64")
    F = np.zeros((n, n))
    F[np.repeat(np.arange(n), np.diff(rp)), ci] = fac
    Mm = (np.tril(F, -1) + np.eye(n)) @ np.triu(F)
    D = np.zeros((n, n))
    D[np.repeat(np.arange(n), np.diff(rp)), ci] = val
    At = D @ np.linalg.inv(Mm)
    At_csr = (n, np.arange(0, n * n + 1, n, dtype=np.int32), np.tile(np.arange(n, dtype=np.int32), n), At.reshape(-1))
    b = inputs.random_vector(n, w, 1, seed=9)
    shadow = oracle.precond(A, fac, b, w, "fp64", 1, True)  # M^-H r0 (x0 = 0)
    two_sided = oracle.krylov("bicg", A, b, w, ilu="fp64", tol_rel=1e-40, maxit=n)
    explicit = oracle.krylov("bicg", At_csr, b, w, tol_rel=1e-40, maxit=n, shadow=shadow)
    k = min(len(two_sided["hist"]), len(explicit["hist"]), 6)
    assert k >= 4
    np.testing.assert_allclose(two_sided["hist"][:k], explicit["hist"][:k], rtol=1e-9)
    plain_shadow = oracle.krylov("bicg", At_csr, b, w, tol_rel=1e-40, maxit=n)
    assert not np.allclose(two_sided["hist"][1:k], plain_shadow["hist"][1:k], rtol=1e-6)  # the shadow matters


@pytest.mark.parametrize("c", [1, 2])
def test_step_invariants(c):
    """Exact-arithmetic invariants of every step, here in QD (rounding ~1e-60): BiCGSTAB's new
    residual is orthogonal to t = A s^ (omega minimises ||s - omega t||), GPBiCG's to c = A t^ and
    to y (the two-term minimisation).  The trace holds the moduli of the normalised inner
    products, so for complex systems a slip in a conjugation (omega from <s, t> instead of
    <t, s>, whose residual is off by a purely imaginary multiple of |t|^2) fails too."""
    n, w = 40, 4
    A = inputs.random_sparse(n, 3, 8, seed=70 + c, complex_=(c == 2), weak_frac=0.0)
    b = inputs.random_vector(n, w, c, seed=10)
    st = oracle.krylov("bicgstab", A, b, w, c, ilu="fp64", tol_rel=1e-50, maxit=60, trace=True)
    assert st["iters"] >= 5
    assert np.max(np.abs(st["trace"][:, 0])) < 1e-50
    gp = oracle.krylov("gpbicg", A, b, w, c, ilu="fp64", tol_rel=1e-50, maxit=60, trace=True)
    assert gp["iters"] >= 5
    assert np.max(np.abs(gp["trace"])) < 1e-50
