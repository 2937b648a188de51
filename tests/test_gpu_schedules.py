"""Every substitution schedule on the GPU against the oracle: the static chunk schedule, the
owner-block schedule per SM (contiguous row blocks, block barriers between levels, shared-memory
values for dependencies inside a block) and per cluster of 8 or 16 SMs (distributed shared memory
between the CTAs of a cluster, cluster barriers) must give the same bits as the oracle for every
factor precision and both orientations (M and M^H), real and complex.  Whole solves and batches
give the same bits under every schedule (checked against the static schedule's solve) and meet
the stated bars of tests/_bars.py against the oracle's runs.  The schedule is forced through
MPK_SUBST_SCHEDULE, which the library reads at each call."""
import numpy as np
import pytest
import torch

import _bars
import oracle
from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

MATS = {
    "convdiff2d": lambda: (inputs.convdiff2d(41, pe=10.0), 1),
    "convdiff3d": lambda: (inputs.convdiff3d(22)[0], 1),
    "random": lambda: (inputs.random_sparse(1500, 3, 15, seed=4), 1),
    "helmholtz": lambda: (inputs.helmholtz2d(29, k=15.0), 2),
    "random_cplx": lambda: (inputs.random_sparse(900, 3, 9, seed=7, complex_=True), 2),
}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(params=["static", "owner", "cluster8", "cluster16"])
def schedule(request, monkeypatch):
    monkeypatch.setenv("MPK_SUBST_SCHEDULE", request.param)
    return request.param


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "mp"])
@pytest.mark.parametrize("trans", [False, True])
def test_precond_both_schedules(schedule, mat, prec, trans):
    A_t, c = MATS[mat]()
    n = A_t[0]
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    for w in (1, 2, 4):
        if prec == "mp" and w == 4 and c == 2:
            continue  # covered by the plain-row tests; slow here
        M = _lib.ILU0(A, "mp", w) if prec == "mp" else _lib.ILU0(A, prec)
        fac = host(M.values()) if prec == "mp" else oracle.ilu0(A_t, prec, c)[1]
        r = inputs.random_vector(n, w, c, seed=70 + w)
        z = host(M.apply(dev(r), w, trans))
        assert M.schedule()[0] == schedule
        ref = oracle.precond(A_t, fac, r, w, prec, c, trans)
        if prec in ("fp32", "bf16") or w <= 2:
            assert np.array_equal(z, ref), (w, np.max(np.abs(z - ref)))
        else:
            assert np.max(np.abs(_bars.mp_diff(z, ref, w))) <= np.max(np.abs(ref)) * 2.0 ** -190


@pytest.mark.parametrize("method", ["bicg", "bicgstab", "gpbicg"])
@pytest.mark.parametrize("ilu", ["fp64", "fp32"])
def test_solves_both_schedules(schedule, method, ilu):
    A_t = inputs.convdiff3d(20)[0]
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    b = oracle.spmv(A_t, inputs.ones(n, w), w)
    M = _lib.ILU0(A, ilu)
    out = _lib.krylov_solve(method, w, A, M, dev(b), tol_rel=1e-25, maxit=400)
    assert M.schedule()[0] == schedule
    with pytest.MonkeyPatch.context() as mp:
        mp.setenv("MPK_SUBST_SCHEDULE", "static")
        base = _lib.krylov_solve(method, w, A, _lib.ILU0(A, ilu), dev(b), tol_rel=1e-25, maxit=400)
    assert out["iters"] == base["iters"] and np.array_equal(out["hist"], base["hist"])
    assert np.array_equal(host(out["x"]), host(base["x"]))
    ref = oracle.krylov(method, A_t, b, w, ilu=ilu, tol_rel=1e-25, maxit=400)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, ilu, w, 1e-25)


def test_batched_owner_schedule(schedule):
    sys_ = [inputs.random_system(n, 800 + n) for n in (700, 1301, 2999)]
    B_t, roff = inputs.block_diagonal(sys_)
    B_t = (B_t[0], B_t[1].astype(np.int32), B_t[2], B_t[3])
    w = 2
    B = _lib.Matrix.from_tuple(B_t)
    b = np.concatenate([oracle.spmv(S, inputs.ones(S[0], w), w) for S in sys_])
    out = _lib.krylov_solve_batched("bicgstab", w, B, roff, _lib.ILU0(B, "fp32"), dev(b), tol_rel=1e-25, maxit=300)
    for k, S in enumerate(sys_):
        ref = oracle.krylov("bicgstab", S, b[roff[k] * w:roff[k + 1] * w], w, ilu="fp32", tol_rel=1e-25, maxit=300)
        assert out["statuses"][k] == ref["status"]
        _bars.check_iters(out["iters"][k], ref["iters"])


def test_auto_tuner_picks_a_schedule(monkeypatch):
    monkeypatch.delenv("MPK_SUBST_SCHEDULE", raising=False)
    A_t = inputs.convdiff3d(32)[0]
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    b = _lib.spmv_mp(A, dev(inputs.ones(n, w)), w)
    M = _lib.ILU0(A, "fp64")
    out = _lib.krylov_solve("bicgstab", w, A, M, b, tol_rel=1e-25)
    sched, wpb = M.schedule()
    assert out["status"] == "OK" and sched in ("static", "owner") and wpb in (4, 8, 16, 32)
    print("tuned schedule at 32^3:", sched, wpb)


@pytest.mark.parametrize("poll", ["lane0", "all", "allsleep"])
@pytest.mark.parametrize("mat", ["convdiff3d", "helmholtz", "random_cplx"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_precond_both_polling_modes(monkeypatch, poll, mat, prec):
    """The substitutions' ways of waiting for dependencies (lane 0 on the chunk's latest one, or
    every lane on its own, spinning or sleeping between rounds) give the oracle's bits, M and M^H
    (the complex binary64 factor runs the paired-warp kernel, real and imaginary parts on two
    sub-partitions), and the handle reports the mode it ran."""
    monkeypatch.setenv("MPK_SUBST_SCHEDULE", "static")
    monkeypatch.setenv("MPK_SUBST_POLL", poll)
    A_t, c = MATS[mat]()
    n = A_t[0]
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    M = _lib.ILU0(A, prec)
    fac = oracle.ilu0(A_t, prec, c)[1]
    for trans in (False, True):
        for w in (1, 2):
            r = inputs.random_vector(n, w, c, seed=90 + w)
            z = host(M.apply(dev(r), w, trans))
            assert np.array_equal(z, oracle.precond(A_t, fac, r, w, prec, c, trans)), (trans, w)
    assert M.polling() == poll
