"""GPU parity of the paper's plain rows (without "_d") against the oracle: the multi-component
ILU(0) (factor entries, products and divisions in the solve's w-component arithmetic), the SpMV
with the matrix promoted to w components, and the Hermitian case of BiCG.
Bars:
  * factor: identical for w <= 2 (the kernel applies the KIJ updates in their sequential order,
    every step the same double-word algorithm); w = 3, 4 within 2^-150 / 2^-200 of the entry's
    magnitude per step count (exact expansions rounded greedily: in practice identical);
  * substitutions M z = r and M^H z = r: identical for w <= 2, w = 3, 4 within 2^-140 / 2^-190 of
    max |z|;
  * Krylov with the factor: the stated bars of tests/_bars.py against the oracle's runs (the
    inner products differ in summation order);
  * a factor built for one w is refused by a solve with another w, and by the learned correction;
  * SpMV with the matrix promoted to w components: identical for w <= 2, within 2^-150 / 2^-200
    for w = 3, 4; whole solves of the plain rows (promoted matrix + multi-component factor),
    single and batched, within the same bars (each batched system identical to its solve alone);
  * Hermitian A: BiCG multiplies A^H p~ by A's own rows (reported), within the same bars.
Sizes span several 32-row chunks and 256-row tiles and end in a ragged tail.
"""
import numpy as np
import pytest
import torch

import _bars
import oracle
from paper_2504_14498_gb300 import _lib, inputs, learned

pytestmark = pytest.mark.gpu

TOL = {3: 2.0 ** -150, 4: 2.0 ** -200}

MATS = {
    "convdiff2d": lambda: (inputs.convdiff2d(41, pe=10.0), 1),
    "convdiff3d": lambda: (inputs.convdiff3d(11)[0], 1),
    "random": lambda: (inputs.random_sparse(1500, 3, 15, seed=4), 1),
    "helmholtz": lambda: (inputs.helmholtz2d(29, k=15.0), 2),
    "random_cplx": lambda: (inputs.random_sparse(900, 3, 9, seed=7, complex_=True), 2),
}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_mp_factor_parity(mat, w):
    A_t, c = MATS[mat]()
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    M = _lib.ILU0(A, "mp", w)
    assert _lib.lib().mpk_ilu0_prec(M.handle) == 3 and _lib.lib().mpk_ilu0_width(M.handle) == w
    got = host(M.values())
    st, ref, _ = oracle.ilu0(A_t, "mp", c, w)
    assert st == 0 and got.shape == ref.shape
    if w <= 2:
        assert np.array_equal(got, ref)
    else:
        r = ref.reshape(-1, c, w)
        err = np.abs(_bars.mp_diff(got, ref, w)).reshape(-1, c)
        mag = np.abs(r[:, :, 0])
        assert np.all(err <= 64 * TOL[w] * np.maximum(mag, np.max(mag) * 2.0 ** -40))


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("w", [1, 2, 3, 4])
@pytest.mark.parametrize("trans", [False, True])
def test_mp_precond_parity(mat, w, trans):
    A_t, c = MATS[mat]()
    n = A_t[0]
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    M = _lib.ILU0(A, "mp", w)
    fac = host(M.values())  # the GPU's factor (identical to the oracle's for w <= 2, see above)
    r = inputs.random_vector(n, w, c, seed=60 + w)
    z = host(M.apply(dev(r), w, trans))
    ref = oracle.precond(A_t, fac, r, w, "mp", c, trans)
    if w <= 2:
        assert np.array_equal(z, ref), np.max(np.abs(z - ref))
    else:
        assert np.max(np.abs(_bars.mp_diff(z, ref, w))) <= np.max(np.abs(ref)) * 2.0 ** (-190 if w == 4 else -140)


def _solve_pair(method, A_t, c, w, tol, maxit=600):
    n = A_t[0]
    xs = inputs.ones(n, w, c)
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    b_ref = oracle.spmv(A_t, xs, w, c)
    M = _lib.ILU0(A, "mp", w)
    out = _lib.krylov_solve(method, w, A, M, dev(b_ref), tol_rel=tol, maxit=maxit)
    ref = oracle.krylov(method, A_t, b_ref, w, c, ilu="mp", tol_rel=tol, maxit=maxit)
    return out, ref


@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
def test_mp_krylov_real_dd(method):
    out, ref = _solve_pair(method, inputs.convdiff2d(33, pe=10.0), 1, 2, 1e-25)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, "mp", 2, 1e-25)
    assert out["relres_true"] < 1e-24 and out["graph"]


@pytest.mark.parametrize("method", ["bicg", "bicgstab", "gpbicg"])
def test_mp_krylov_complex_dd(method):
    out, ref = _solve_pair(method, inputs.helmholtz2d(23, k=10.0), 2, 2, 1e-25)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, "mp", 2, 1e-25, indefinite=True)


@pytest.mark.parametrize("w,tol", [(3, 1e-40), (4, 1e-55)])
def test_mp_krylov_td_qd(w, tol):
    out, ref = _solve_pair("bicgstab", inputs.convdiff2d(14, pe=10.0), 1, w, tol)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, "mp", w, tol)


def test_mp_factor_same_iterations_as_binary64_factor():
    """Table 1: the multi-component factor and the binary64 factor need the same number of
    iterations (to within one) on the real test problem; checked here on the GPU."""
    A_t = inputs.convdiff2d(40, pe=10.0)
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    b = _lib.spmv_mp(A, dev(inputs.ones(n, w)), w)
    a = _lib.krylov_solve("bicgstab", w, A, _lib.ILU0(A, "mp", w), b)
    d = _lib.krylov_solve("bicgstab", w, A, _lib.ILU0(A, "fp64"), b)
    assert a["status"] == d["status"] == "OK"
    assert abs(a["iters"] - d["iters"]) <= 1


def test_mp_factor_errors():
    A_t = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 1.0, 1.0, 1.0]))
    with pytest.raises(_lib.MpkError) as e:
        _lib.ILU0(_lib.Matrix.from_tuple(A_t), "mp", 2)
    assert e.value.status == "ZERO_PIVOT"
    st, _, fr = oracle.ilu0(A_t, "mp", 1, 2)
    assert st == 3 and fr == 1
    C_t = inputs.convdiff2d(12, pe=5.0)
    C = _lib.Matrix.from_tuple(C_t)
    M = _lib.ILU0(C, "mp", 2)
    r = dev(inputs.random_vector(C_t[0], 3, 1, seed=2))
    with pytest.raises(_lib.MpkError) as e:
        M.apply(r, 3)
    assert e.value.status == "INVALID_ARG"
    b = _lib.spmv_mp(C, dev(inputs.ones(C_t[0], 4)), 4)
    with pytest.raises(_lib.MpkError) as e:
        _lib.krylov_solve("bicgstab", 4, C, M, b)
    assert e.value.status == "INVALID_ARG"
    with pytest.raises(_lib.MpkError) as e:
        learned.LearnedILU(seed=1).correct(C, M)
    assert e.value.status == "INVALID_ARG"
    with pytest.raises(_lib.MpkError) as e:
        _lib.ILU0(C, "mp", 5)
    assert e.value.status == "INVALID_ARG"


def test_mp_solve_host_end_to_end():
    A_t = inputs.convdiff2d(30, pe=10.0)
    n, w = A_t[0], 2
    b = oracle.spmv(A_t, inputs.ones(n, w), w)
    out = _lib.solve_host("bicgstab", w, "mp", A_t, b, tol_rel=1e-25)
    ref = oracle.krylov("bicgstab", A_t, b, w, ilu="mp", tol_rel=1e-25)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_iters(out["iters"], ref["iters"])
    assert _bars.rel_error(out["x"], inputs.ones(n, w), n, 1, w) <= 1e-24


# ---- SpMV with the matrix promoted to w components (the rows without "_d") ----------------------

@pytest.mark.parametrize("c", [1, 2])
@pytest.mark.parametrize("w", [1, 2, 3, 4])
def test_mp_matrix_spmv_parity(w, c):
    A_t = inputs.random_sparse(3001, 3, 20, seed=91) if c == 1 else inputs.random_sparse(2003, 3, 12, seed=92,
                                                                                        complex_=True)
    n = A_t[0]
    x = inputs.random_vector(n, w, c, seed=27 + w)
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    y = host(_lib.spmv_mp(A, dev(x), w, mp_matrix=True))
    ref = oracle.spmv(A_t, x, w, c, mp_matrix=True)
    if w <= 2:
        assert np.array_equal(y, ref)
    else:
        lead = np.abs(ref.reshape(n, c, w)[:, :, 0])
        err = np.abs(_bars.mp_diff(y, ref, w)).reshape(n, c)
        assert np.all(err <= TOL[w] * 64 * np.maximum(lead, np.max(lead) * 2.0 ** -30))


@pytest.mark.parametrize("method", ["bicg", "cgs", "bicgstab", "gpbicg"])
def test_plain_rows(method):
    """The paper's plain rows ("BiCG_ILU(0)" etc.): promoted matrix and multi-component factor."""
    A_t = inputs.convdiff2d(33, pe=10.0)
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    b_ref = oracle.spmv(A_t, inputs.ones(n, w), w)
    out = _lib.krylov_solve(method, w, A, _lib.ILU0(A, "mp", w), dev(b_ref), tol_rel=1e-25, maxit=600, mp_matrix=True)
    ref = oracle.krylov(method, A_t, b_ref, w, ilu="mp", tol_rel=1e-25, maxit=600, mp_matrix=True)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, "mp", w, 1e-25)
    assert out["relres_true"] <= 1e-24


def test_plain_rows_batched():
    sys_ = [inputs.convdiff2d_random(m, 300 + m) for m in (12, 17, 23)]
    B_t, roff = inputs.block_diagonal(sys_)
    B_t = (B_t[0], B_t[1].astype(np.int32), B_t[2], B_t[3])
    w = 2
    B = _lib.Matrix.from_tuple(B_t)
    b = np.concatenate([oracle.spmv(S, inputs.ones(S[0], w), w) for S in sys_])
    out = _lib.krylov_solve_batched("bicgstab", w, B, roff, _lib.ILU0(B, "mp", w), dev(b), tol_rel=1e-25, maxit=400,
                                    mp_matrix=True)
    x = host(out["x"])
    for k, S in enumerate(sys_):
        bk = b[roff[k] * w:roff[k + 1] * w]
        As = _lib.Matrix.from_tuple(S)
        one = _lib.krylov_solve("bicgstab", w, As, _lib.ILU0(As, "mp", w), dev(bk), tol_rel=1e-25, maxit=400,
                                mp_matrix=True)
        assert out["iters"][k] == one["iters"] and np.array_equal(x[roff[k] * w:roff[k + 1] * w], host(one["x"]))
        ref = oracle.krylov("bicgstab", S, bk, w, ilu="mp", tol_rel=1e-25, maxit=400, mp_matrix=True)
        assert out["statuses"][k] == ref["status"] == "OK"
        _bars.check_iters(out["iters"][k], ref["iters"])


# ---- Hermitian systems ------------------------------------------------------------------------

@pytest.mark.parametrize("ilu", ["fp64", "mp"])
def test_hermitian_bicg_reuses_A(ilu):
    A_t = inputs.magnetic_laplacian2d(31)
    n, w, c = A_t[0], 2, 2
    A = _lib.Matrix.from_tuple(A_t, is_complex=True)
    b_ref = oracle.spmv(A_t, inputs.ones(n, w, c), w, c)
    M = _lib.ILU0(A, ilu, w) if ilu == "mp" else _lib.ILU0(A, ilu)
    out = _lib.krylov_solve("bicg", w, A, M, dev(b_ref), tol_rel=1e-25, maxit=600)
    ref = oracle.krylov("bicg", A_t, b_ref, w, c, ilu=ilu, tol_rel=1e-25, maxit=600)
    assert out["hermitian"]  # q~ = A^H p~ multiplied by A's own rows: no transpose built
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, ilu, w, 1e-25)


def test_non_hermitian_bicg_builds_transpose():
    A_t = inputs.helmholtz2d(23, k=10.0)  # complex symmetric, not Hermitian
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t, is_complex=True)
    b = _lib.spmv_mp(A, dev(inputs.ones(n, w, 2)), w)
    out = _lib.krylov_solve("bicg", w, A, _lib.ILU0(A, "fp64"), b, tol_rel=1e-20, maxit=300)
    assert not out["hermitian"] and out["status"] == "OK"
    # a real symmetric matrix is Hermitian
    S_t = inputs.tridiag(300, -1.0, 2.5, -1.0)
    S = _lib.Matrix.from_tuple(S_t)
    bs = _lib.spmv_mp(S, dev(inputs.ones(300, w)), w)
    o2 = _lib.krylov_solve("bicg", w, S, _lib.ILU0(S, "fp64"), bs, tol_rel=1e-25, maxit=300)
    assert o2["hermitian"] and o2["status"] == "OK"
