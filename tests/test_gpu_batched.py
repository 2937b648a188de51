"""Batched solves (many independent systems in the same launches).  Every system of a batch
performs the operation sequence of its own solve, so each system's iterations, residual history
and iterate are identical to the library's solve of that system alone (checked bit for bit), and
against the oracle's run of the system they meet the stated bars (tests/_bars.py); statuses are
per system (converged, breakdown, iteration limit, b = 0).
"""
import numpy as np
import pytest
import torch

import _bars
import oracle
from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _batch(sizes, seed0, extra=()):
    systems = [inputs.random_system(int(n), seed0 + k) for k, n in enumerate(sizes)] + list(extra)
    A_t, roff = inputs.block_diagonal(systems)
    A_t = (A_t[0], A_t[1].astype(np.int32), A_t[2], A_t[3])
    return systems, A_t, roff


def _rhs(systems, w, seed0):
    xs = [inputs.batch_xstar(S[0], w, seed0 + k) for k, S in enumerate(systems)]
    bs = [oracle.spmv(S, x, w) for S, x in zip(systems, xs)]
    return xs, bs


def _check_against_oracle(method, w, ilu, systems, roff, out, bs, tol, maxit, c=1, indefinite=False):
    """Every system: identical to the library's solve of it alone, and within the stated bars of
    the oracle's run."""
    x = host(out["x"])
    for k, S in enumerate(systems):
        As = _lib.Matrix.from_tuple(S, is_complex=(c == 2))
        one = _lib.krylov_solve(method, w, As, _lib.ILU0(As, ilu) if ilu != "none" else None, dev(bs[k]),
                                tol_rel=tol, maxit=maxit)
        assert out["statuses"][k] == one["status"] and out["iters"][k] == one["iters"], k
        assert np.array_equal(out["hist"][k], one["hist"]), k
        assert np.array_equal(x[roff[k] * c * w:roff[k + 1] * c * w], host(one["x"])), k
        assert out["relres_true"][k] == one["relres_true"] and out["replacements"][k] == one["replacements"], k
        ref = oracle.krylov(method, S, bs[k], w, c, ilu=ilu, tol_rel=tol, maxit=maxit)
        got = {"status": out["statuses"][k], "iters": int(out["iters"][k]), "hist": out["hist"][k]}
        _bars.check_solve(got, ref, ilu, w, tol, indefinite=indefinite)
        if got["status"] == "OK":
            assert out["relres_true"][k] <= 10 * tol


@pytest.mark.parametrize("method", ["bicgstab", "gpbicg", "cgs", "bicg"])
@pytest.mark.parametrize("ilu", ["fp32", "fp64"])
def test_batched_equals_separate_solves(method, ilu):
    systems, A_t, roff = _batch([1000, 257, 3001, 640, 1999, 33], 900 + len(method))
    w, tol, maxit = 2, 1e-25, 400
    xs, bs = _rhs(systems, w, 77)
    A = _lib.Matrix.from_tuple(A_t)
    M = _lib.ILU0(A, ilu)
    out = _lib.krylov_solve_batched(method, w, A, roff, M, dev(np.concatenate(bs)), tol_rel=tol, maxit=maxit,
                                    check_every=7, history=True)
    _check_against_oracle(method, w, ilu, systems, roff, out, bs, tol, maxit)
    assert all(s == "OK" for s in out["statuses"])


def test_batched_mixed_statuses():
    # a system with b = 0 (done before the first iteration), a 2x2 system that breaks down, and
    # ordinary systems with different iteration counts; the iteration limit stops the slowest
    br = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([0.0, 1.0, 1.0, 0.0]))
    systems, A_t, roff = _batch([500, 800, 1200], 31, extra=[br])
    w, tol, maxit = 2, 1e-25, 9
    xs, bs = _rhs(systems, w, 5)
    bs[1] = np.zeros_like(bs[1])
    bs[3] = np.array([1.0, 0.0, 0.0, 0.0])
    A = _lib.Matrix.from_tuple(A_t)
    out = _lib.krylov_solve_batched("bicgstab", w, A, roff, None, dev(np.concatenate(bs)), tol_rel=tol,
                                    maxit=maxit, check_every=4, history=True)
    _check_against_oracle("bicgstab", w, "none", systems, roff, out, bs, tol, maxit)
    assert out["statuses"][1] == "OK" and out["iters"][1] == 0
    assert out["statuses"][3] == "BREAKDOWN"
    assert "MAXIT" in out["statuses"]


def test_batched_complex_and_qd():
    sys_c = [inputs.helmholtz2d(m, k=10.0) for m in (9, 17, 23)]
    A_t, roff = inputs.block_diagonal(sys_c)
    A_t = (A_t[0], A_t[1].astype(np.int32), A_t[2], A_t[3])
    w = 2
    bs = [oracle.spmv(S, inputs.random_vector(S[0], w, 2, seed=3 + k), w, 2) for k, S in enumerate(sys_c)]
    A = _lib.Matrix.from_tuple(A_t, is_complex=True)
    M = _lib.ILU0(A, "fp32")
    out = _lib.krylov_solve_batched("bicgstab", w, A, roff, M, dev(np.concatenate(bs)), tol_rel=1e-25, maxit=300,
                                    history=True)
    _check_against_oracle("bicgstab", w, "fp32", sys_c, roff, out, bs, 1e-25, 300, c=2, indefinite=True)
    systems, A_t, roff = _batch([300, 700], 44)
    xs, bs = _rhs(systems, 4, 9)
    A = _lib.Matrix.from_tuple(A_t)
    out = _lib.krylov_solve_batched("bicgstab", 4, A, roff, _lib.ILU0(A, "fp64"), dev(np.concatenate(bs)),
                                    tol_rel=1e-55, maxit=300, history=True)
    _check_against_oracle("bicgstab", 4, "fp64", systems, roff, out, bs, 1e-55, 300)
    assert all(s == "OK" for s in out["statuses"])


def test_batched_rejects_cross_block_columns():
    systems, A_t, roff = _batch([40, 50], 3)
    n, rp, ci, val = A_t
    ci = ci.copy()
    ci[rp[5] + 1] = roff[1] + 3  # row 5 (system 0) gets a column in system 1
    ci[rp[5]:rp[6]] = np.sort(ci[rp[5]:rp[6]])
    A = _lib.Matrix.from_tuple((n, rp, ci, val))
    with pytest.raises(_lib.MpkError) as e:
        _lib.krylov_solve_batched("bicgstab", 2, A, roff, None, dev(np.ones(2 * n)), maxit=5)
    assert e.value.status == "INVALID_ARG"


def test_batch_512_full_size():
    """The batched workload at full size: 512 systems, N log-uniform in [1k, 200k] (20.4M rows),
    binary32 ILU(0), DD BiCGSTAB to 1e-25 in one batched solve.  Every system must reach the
    tolerance with a small true residual; the three smallest systems and a median one are compared
    with the library's solves of them alone (bit for bit) and with the oracle's runs (stated
    bars)."""
    sizes = inputs.batch_sizes()
    systems = [inputs.batch_system(s, sizes) for s in range(len(sizes))]
    A_t, roff = inputs.block_diagonal(systems)
    A_t = (A_t[0], A_t[1].astype(np.int32), A_t[2], A_t[3])
    w = 2
    pick = list(np.argsort(sizes)[:3]) + [int(np.argsort(sizes)[len(sizes) // 2])]
    bs = {}
    for s in range(len(sizes)):
        xs = inputs.batch_xstar(int(sizes[s]), w, 2504_14498 + 9000 + s)
        if s in pick:
            bs[s] = oracle.spmv(systems[s], xs, w)
    del systems
    A = _lib.Matrix.from_tuple(A_t)
    xstar = dev(np.concatenate([inputs.batch_xstar(int(sizes[s]), w, 2504_14498 + 9000 + s)
                                for s in range(len(sizes))]))
    bd = _lib.spmv_mp(A, xstar, w)
    M = _lib.ILU0(A, "fp32")
    out = _lib.krylov_solve_batched("bicgstab", w, A, roff, M, bd, tol_rel=1e-25, maxit=2000, check_every=10)
    assert all(s == "OK" for s in out["statuses"]), [s for s in out["statuses"] if s != "OK"][:5]
    assert np.all(out["relres_true"] < 1e-23)
    x = host(out["x"])
    bh = host(bd)
    for s in pick:
        S = inputs.batch_system(s, sizes)
        assert np.array_equal(bh[roff[s] * w:roff[s + 1] * w], bs[s])
        As = _lib.Matrix.from_tuple(S)
        one = _lib.krylov_solve("bicgstab", w, As, _lib.ILU0(As, "fp32"), dev(bs[s]), tol_rel=1e-25, maxit=2000)
        assert out["iters"][s] == one["iters"] and out["statuses"][s] == one["status"]
        assert np.array_equal(x[roff[s] * w:roff[s + 1] * w], host(one["x"]))
        ref = oracle.krylov("bicgstab", S, bs[s], w, ilu="fp32", tol_rel=1e-25, maxit=2000)
        assert ref["status"] == "OK"
        _bars.check_iters(out["iters"][s], ref["iters"])
