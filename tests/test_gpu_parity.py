"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs.  Bars (from the statement of the method's tolerances):
  * mixed SpMV: identical to the oracle for D and DD (same operations in the same CSR order);
    TD / QD within 2^-150 / 2^-200 of sum_j |a_ij||x_j| per row (and in practice identical);
  * inner products: within 2^-100 (DD), 2^-150 (TD), 2^-200 (QD) of sum |a_i b_i| (D: 4 n u) of
    the oracle's left-to-right sum, since the GPU reduces in a fixed tree order; that order is
    checked bit for bit separately (determinism, tests/_tree_dot.py);
  * ILU(0) factors: identical (<= 2 ulp asked; the kernel follows the KIJ update order exactly);
  * substitutions: identical for binary32 / bfloat16 factors and for D / DD vectors;
  * Krylov (tests/_bars.py): residual norms within 1e-10 relative over the first 20 iterations
    above the floor stated there, iteration count within 5 % (at least 1), the same status, the
    true residual within 10x the target, and on well-conditioned systems solved to 1e-31 (DD) /
    1e-63 (QD) a final error <= 1e-28 / 1e-60 against x*.
Sizes span several 256-row tiles and end in a ragged tail.
"""
import numpy as np
import pytest
import torch

import _bars
import _tree_dot
import oracle
from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

TOL = {2: 2.0 ** -100, 3: 2.0 ** -150, 4: 2.0 ** -200}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _row_mag(A, x, w, c):
    """sum_j |a_ij| |x_j| per row and part (leading components suffice for a tolerance)."""
    n, rp, ci, val = A
    X = np.abs(x.reshape(-1, c, w)[:, :, 0])
    if c == 1:
        av = np.abs(val)
        return np.add.reduceat(av * X[ci, 0], rp[:-1]).reshape(n, 1) if len(ci) else np.zeros((n, 1))
    ar, ai = np.abs(val[0::2]), np.abs(val[1::2])
    m = (ar + ai) * (X[ci, 0] + X[ci, 1])
    s = np.add.reduceat(m, rp[:-1])
    return np.stack([s, s], axis=1)


MATS = {
    "random_real": lambda: (inputs.random_sparse(3001, 3, 20, seed=91), 1),
    "random_cplx": lambda: (inputs.random_sparse(2003, 3, 12, seed=92, complex_=True), 2),
    "convdiff3d": lambda: (inputs.convdiff3d(13)[0], 1),
    "helmholtz": lambda: (inputs.helmholtz2d(37, k=12.0), 2),
}


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_spmv_parity(mat, w):
    A_t, c = MATS[mat]()
    n = A_t[0]
    x = inputs.random_vector(n, w, c, seed=17 + w)
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    y = host(_lib.spmv_mp(A, dev(x), w))
    ref = oracle.spmv(A_t, x, w, c)
    if w <= 2:
        assert np.array_equal(y, ref)
    else:
        err = np.abs(_bars.mp_diff(y, ref, w)).reshape(n, c)
        assert np.all(err <= TOL[w] * _row_mag(A_t, x, w, c) * 4)


@pytest.mark.parametrize("w", [1, 2, 3, 4])
@pytest.mark.parametrize("c", [1, 2])
@pytest.mark.parametrize("n", [1, 17, 255, 4097, 70001, 1048577])
def test_dot_parity(w, c, n):
    a = inputs.random_vector(n, w, c, seed=5)
    b = inputs.random_vector(n, w, c, seed=6)
    got = host(_lib.dot(dev(a), dev(b), n, w, c == 2)).reshape(c, w)
    ref = oracle.dot(a, b, n, w, c).reshape(c, w)
    if n <= 70001 and w <= 2:  # determinism: the kernel's fixed tree order, bit for bit
        assert np.array_equal(got.ravel(), _tree_dot.tree_dot(a, b, n, w, c))
    elif w > 2:  # TD / QD: the device arithmetic is not the oracle's exact one; same bits on a rerun
        assert np.array_equal(got, host(_lib.dot(dev(a), dev(b), n, w, c == 2)).reshape(c, w))
    A, B = a.reshape(n, c, w)[:, :, 0], b.reshape(n, c, w)[:, :, 0]
    mag = np.sum(np.abs(A).sum(axis=1) * np.abs(B).sum(axis=1))
    tol = TOL[w] * 8 if w > 1 else 4 * n * 2.0 ** -53
    for part in range(c):
        assert abs(got[part].sum() - ref[part].sum()) <= tol * mag + abs(ref[part, 0]) * 2.0 ** (-53 * w + 2)


ILU_MATS = {
    "convdiff2d": lambda: (inputs.convdiff2d(41, pe=10.0), 1),
    "convdiff3d": lambda: (inputs.convdiff3d(11)[0], 1),
    "random": lambda: (inputs.random_sparse(1500, 3, 15, seed=4), 1),
    "helmholtz": lambda: (inputs.helmholtz2d(29, k=15.0), 2),
    "random_cplx": lambda: (inputs.random_sparse(900, 3, 9, seed=7, complex_=True), 2),
}


@pytest.mark.parametrize("mat", list(ILU_MATS))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_ilu0_bitwise(mat, prec):
    A_t, c = ILU_MATS[mat]()
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    M = _lib.ILU0(A, prec)
    got = host(M.values())
    st, ref, _ = oracle.ilu0(A_t, prec, c)
    assert st == 0
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mat", list(ILU_MATS))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("trans", [False, True])
def test_precond_parity(mat, prec, trans):
    A_t, c = ILU_MATS[mat]()
    n = A_t[0]
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    M = _lib.ILU0(A, prec)
    _, fac, _ = oracle.ilu0(A_t, prec, c)
    for w in (1, 2, 4):
        r = inputs.random_vector(n, w, c, seed=40 + w)
        z = host(M.apply(dev(r), w, trans))
        ref = oracle.precond(A_t, fac, r, w, prec, c, trans)
        if prec != "fp64" or w <= 2:
            assert np.array_equal(z, ref), (w, np.max(np.abs(z - ref)))
        else:
            scale = np.max(np.abs(ref))
            assert np.max(np.abs(_bars.mp_diff(z, ref, w))) <= scale * 2.0 ** -190


def test_ilu0_errors_reported():
    A_t = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 1.0, 1.0, 1.0]))
    with pytest.raises(_lib.MpkError) as e:
        _lib.ILU0(_lib.Matrix.from_tuple(A_t), "fp64")
    assert e.value.status == "ZERO_PIVOT"
    B_t = (2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    with pytest.raises(_lib.MpkError) as e:
        _lib.ILU0(_lib.Matrix.from_tuple(B_t), "fp64")
    assert e.value.status == "MISSING_DIAG"
    C_t = (2, np.array([0, 2, 3], np.int32), np.array([1, 0, 1], np.int32), np.array([1.0, 2.0, 3.0]))
    with pytest.raises(_lib.MpkError) as e:
        _lib.ILU0(_lib.Matrix.from_tuple(C_t), "fp64")
    assert e.value.status == "INVALID_ARG"


def _compare_solve(method, A_t, c, w, ilu, tol, maxit=600, x_star=None, indefinite=False, **kw):
    n = A_t[0]
    xs = inputs.ones(n, w, c) if x_star is None else x_star
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    b_dev = _lib.spmv_mp(A, dev(xs), w)
    b_ref = oracle.spmv(A_t, xs, w, c)
    assert np.array_equal(host(b_dev), b_ref) or w > 2
    M = _lib.ILU0(A, ilu) if ilu != "none" else None
    out = _lib.krylov_solve(method, w, A, M, b_dev, tol_rel=tol, maxit=maxit, **kw)
    ref = oracle.krylov(method, A_t, b_ref, w, c, ilu=ilu, tol_rel=tol, maxit=maxit, **kw)
    _bars.check_solve(out, ref, ilu, w, tol, indefinite=indefinite)
    if out["status"] == "OK" and kw.get("true_res_period", _lib.TRUE_RES_PERIOD) > 0:
        assert out["relres_true"] <= 10 * tol  # the replacement rule's acceptance level
    assert out["graph"]  # the iterations ran as replays of one captured CUDA graph
    return out, ref


@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
def test_stopping_rule_absolute_term(method):
    """||r_k|| < eps_r ||r_0|| + eps_a with the absolute term deciding (eps_r = 0, and both
    terms): the GPU stops at the first norm below the threshold, at the oracle's iteration."""
    A_t = inputs.convdiff2d(10, pe=10.0)
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    b_ref = oracle.spmv(A_t, inputs.ones(n, w), w)
    M = _lib.ILU0(A, "fp64")
    r0 = oracle.krylov(method, A_t, b_ref, w, ilu="fp64", maxit=1)["hist"][0]
    for tol_rel, tol_abs in ((0.0, 1e-6 * r0), (1e-9, 1e-6 * r0)):
        out = _lib.krylov_solve(method, w, A, M, dev(b_ref), tol_rel=tol_rel, tol_abs=tol_abs, maxit=200)
        ref = oracle.krylov(method, A_t, b_ref, w, ilu="fp64", tol_rel=tol_rel, tol_abs=tol_abs, maxit=200)
        assert out["status"] == ref["status"] == "OK"
        thr = tol_rel * out["hist"][0] + tol_abs
        assert out["hist"][-1] < thr and np.all(out["hist"][:-1] >= thr)
        _bars.check_band(out["hist"], ref["hist"], _bars.band_floor("fp64", w))
        assert out["iters"] == ref["iters"]


@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
@pytest.mark.parametrize("ilu", ["fp64", "fp32", "bf16", "none"])
def test_krylov_real_dd(method, ilu):
    """Unpreconditioned runs compare the plain method (no replacement): after a replacement their
    remaining lengths depend on the rounding of the true residual they restart from (measured:
    up to 50 % apart between two valid summation orders); the rule itself is checked below."""
    A_t = inputs.convdiff2d(33, pe=10.0)
    kw = {"true_res_period": 0} if ilu == "none" else {}
    out, ref = _compare_solve(method, A_t, 1, 2, ilu, 1e-25, maxit=3000 if ilu == "none" else 600, **kw)
    assert out["status"] == "OK"
    if ilu != "none":
        assert out["relres_true"] < 1e-24


@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
@pytest.mark.parametrize("ilu", ["fp64", "fp32"])
def test_krylov_complex_dd(method, ilu):
    """Indefinite system: band over 12 iterations, iteration counts within 20 % (tests/_bars.py).
    CGS with the replacement rule stagnates on this system on both sides: replacing r alone leaves
    CGS's u, p, q built on the old r; its plain run (period 0) converges."""
    A_t = inputs.helmholtz2d(23, k=10.0)
    kw = {"true_res_period": 0} if method == "cgs" else {}
    out, ref = _compare_solve(method, A_t, 2, 2, ilu, 1e-25, indefinite=True, **kw)
    if (method, ilu) != ("cgs", "fp32"):  # CGS stagnates with the binary32 factor on this indefinite
        assert out["status"] == "OK" and out["relres_true"] < 1e-24  # system, on both sides


@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
@pytest.mark.parametrize("ilu", ["none", "fp64", "fp32"])
def test_replacement_parity(method, ilu):
    """The replacement rule with a short period (5): checks at the same iterations, the same
    number of replacements, the true norms at the checks within 1e-10 above the band floor."""
    A_t = inputs.convdiff2d(33, pe=10.0)
    out, ref = _compare_solve(method, A_t, 1, 2, ilu, 1e-25, maxit=3000, true_res_period=5)
    assert out["status"] == "OK" and out["replacements"] == ref["replacements"] >= 1
    floor = _bars.band_floor(ilu, 2)
    r0 = ref["hist"][0]
    for k in range(1, min(21, len(ref["hist_true"]), len(out["hist_true"]))):
        g, r = out["hist_true"][k], ref["hist_true"][k]
        assert np.isnan(g) == np.isnan(r), k
        if not np.isnan(r) and r >= floor * r0 and ref["hist"][k] >= floor * r0:
            assert abs(g - r) <= 1e-10 * r, (k, g, r)


def test_replacement_guards_false_convergence():
    """Unpreconditioned DD CGS: without the rule the recursive residual passes 1e-25 while the
    true one is ~1e-6 (both sides); with period 50 the solve ends within 10x the target."""
    A_t = inputs.convdiff2d(33, pe=10.0)
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    b = _lib.spmv_mp(A, dev(inputs.ones(n, w)), w)
    plain = _lib.krylov_solve("cgs", w, A, None, b, tol_rel=1e-25, maxit=3000, true_res_period=0)
    assert plain["status"] == "OK" and plain["relres_true"] > 1e-12 and plain["replacements"] == 0
    ruled = _lib.krylov_solve("cgs", w, A, None, b, tol_rel=1e-25, maxit=3000, true_res_period=50)
    assert ruled["status"] == "OK" and ruled["relres_true"] <= 1e-24 and ruled["replacements"] >= 1
    k = ruled["iters"]
    assert ruled["hist_true"][k] == pytest.approx(ruled["relres_true"] * ruled["res0"], rel=1e-12)
    ref = oracle.krylov("cgs", A_t, host(b), w, ilu="none", tol_rel=1e-25, maxit=3000, true_res_period=50)
    assert ref["status"] == "OK" and ref["relres_true"] <= 1e-24 and ref["replacements"] >= 1


WELL = {
    "random_real": lambda: (inputs.random_sparse(3001, 3, 20, seed=91), 1),
    "random_cplx": lambda: (inputs.random_sparse(2003, 3, 12, seed=92, complex_=True), 2),
    "convdiff2d": lambda: (inputs.convdiff2d(33, pe=10.0), 1),
}


@pytest.mark.parametrize("mat", list(WELL))
@pytest.mark.parametrize("ilu", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("w,tol,bound", [(2, 1e-31, 1e-28), (4, 1e-63, 1e-60)])
def test_final_error_well_conditioned(mat, ilu, w, tol, bound):
    """Well-conditioned systems solved to 1e-31 (DD) / 1e-63 (QD): final error against a random
    x* within 1e-28 / 1e-60, and the stated bars against the oracle's run."""
    A_t, c = WELL[mat]()
    n = A_t[0]
    xs = inputs.random_vector(n, w, c, seed=123)
    out, ref = _compare_solve("bicgstab", A_t, c, w, ilu, tol, maxit=600, x_star=xs)
    assert out["status"] == "OK"
    assert _bars.rel_error(host(out["x"]), xs, n, c, w) <= bound
    assert _bars.rel_error(ref["x"], xs, n, c, w) <= bound


@pytest.mark.parametrize("method", ["bicgstab", "gpbicg", "bicg", "cgs"])
@pytest.mark.parametrize("w,tol", [(1, 1e-13), (3, 1e-40), (4, 1e-55)])
def test_krylov_other_precisions(method, w, tol):
    A_t = inputs.convdiff2d(14, pe=10.0)
    out, ref = _compare_solve(method, A_t, 1, w, "fp64", tol)
    assert out["status"] == "OK"


def test_gpbicg_eta0_reduces_to_bicgstab_on_gpu():
    A_t = inputs.convdiff2d(20, pe=5.0)
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    b = _lib.spmv_mp(A, dev(inputs.ones(n, w)), w)
    M = _lib.ILU0(A, "fp64")
    g = _lib.krylov_solve("gpbicg", w, A, M, b, force_eta0=True)
    s = _lib.krylov_solve("bicgstab", w, A, M, b)
    k = min(12, len(g["hist"]), len(s["hist"]))
    np.testing.assert_allclose(g["hist"][:k], s["hist"][:k], rtol=1e-12)


def test_krylov_statuses():
    A_t = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([0.0, 1.0, 1.0, 0.0]))
    A = _lib.Matrix.from_tuple(A_t)
    b = dev(np.array([1.0, 0.0, 0.0, 0.0]))
    for m in ("bicg", "cgs", "bicgstab", "gpbicg"):
        assert _lib.krylov_solve(m, 2, A, None, b, maxit=10)["status"] == "BREAKDOWN"
    C_t = inputs.convdiff2d(10, pe=10.0)
    C = _lib.Matrix.from_tuple(C_t)
    bb = _lib.spmv_mp(C, dev(inputs.ones(C_t[0], 2)), 2)
    out = _lib.krylov_solve("bicgstab", 2, C, None, bb, maxit=3)
    assert out["status"] == "MAXIT" and out["iters"] == 3
    bn = bb.clone()
    bn[10] = float("nan")
    assert _lib.krylov_solve("bicgstab", 2, C, _lib.ILU0(C, "fp64"), bn)["status"] == "NAN"
    zero = torch.zeros_like(bb)
    out = _lib.krylov_solve("bicgstab", 2, C, None, zero)
    assert out["status"] == "OK" and out["iters"] == 0


def test_solve_host_end_to_end():
    A_t = inputs.convdiff2d(30, pe=10.0)
    n, w = A_t[0], 2
    b = host(_lib.spmv_mp(_lib.Matrix.from_tuple(A_t), dev(inputs.ones(n, w)), w))
    out = _lib.solve_host("bicgstab", w, "fp32", A_t, b, tol_rel=1e-25)
    ref = oracle.krylov("bicgstab", A_t, oracle.spmv(A_t, inputs.ones(n, w), w), w, ilu="fp32", tol_rel=1e-25)
    assert out["status"] == "OK"
    assert abs(out["iters"] - ref["iters"]) <= max(1, int(0.05 * ref["iters"]))
    assert np.max(np.abs(out["x"].reshape(n, w)[:, 0] - 1.0)) < 1e-20


def test_solve_host_pinned_in_place():
    """The host-buffer call with page-locked inputs and x returned into x0's own buffer gives the
    bits of the copying call."""
    A_t = inputs.convdiff2d(30, pe=10.0)
    n, w = A_t[0], 2
    b = host(_lib.spmv_mp(_lib.Matrix.from_tuple(A_t), dev(inputs.ones(n, w)), w))
    ref = _lib.solve_host("bicgstab", w, "fp64", A_t, b, tol_rel=1e-25)

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    Ap = (A_t[0], pinned(A_t[1].astype(np.int32)), pinned(A_t[2].astype(np.int32)), pinned(A_t[3]))
    x0 = pinned(np.zeros(n * w))
    out = _lib.solve_host("bicgstab", w, "fp64", Ap, pinned(b), x0, tol_rel=1e-25, x_inplace=True)
    assert out["x"] is x0
    assert out["status"] == ref["status"] == "OK" and out["iters"] == ref["iters"]
    assert np.array_equal(x0, ref["x"])


def test_misaligned_vectors_refused():
    """A vector view that is not 16-byte aligned (offset by one binary64 word) is refused with
    INVALID_ARG before any launch; the aligned call on the same data works."""
    A_t = inputs.convdiff2d(8, pe=1.0)
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    buf = torch.zeros(n * w + 2, dtype=torch.float64, device="cuda")
    x = dev(inputs.ones(n, w))
    with pytest.raises(_lib.MpkError) as e:
        _lib.spmv_mp(A, x, w, buf[1:1 + n * w])
    assert e.value.status == "INVALID_ARG"
    y = _lib.spmv_mp(A, x, w, buf[2:2 + n * w])
    assert np.array_equal(host(y), oracle.spmv(A_t, inputs.ones(n, w), w))
