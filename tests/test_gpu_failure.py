"""Failure detection on the GPU without a fault: a substitution whose dependency is never
published (the testing aid mpk_ilu0_test_withhold) must end by its bounded waits (about a
second), report MPK_TIMEOUT once, and leave the handle and the context usable: the next call on
the same handle returns the same bits as before."""
import time

import numpy as np
import pytest
import torch

from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("schedule", ["static", "owner"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_withheld_row_times_out_and_handle_recovers(schedule, prec, monkeypatch):
    monkeypatch.setenv("MPK_SUBST_SCHEDULE", schedule)
    A_t = inputs.convdiff2d(40, pe=10.0)
    n, w = A_t[0], 2
    A = _lib.Matrix.from_tuple(A_t)
    M = _lib.ILU0(A, prec)
    r = dev(inputs.random_vector(n, w, 1, seed=3))
    z_ok = host(M.apply(r, w))
    M.test_withhold(0)  # row 0 starts the lower triangle's dependency chain
    t0 = time.time()
    with pytest.raises(_lib.MpkError) as e:
        M.apply(r, w)
    assert e.value.status == "TIMEOUT"
    assert time.time() - t0 < 60
    M.test_withhold(-1)
    assert np.array_equal(host(M.apply(r, w)), z_ok)  # reported once; the handle serves again
    b = _lib.spmv_mp(A, dev(inputs.ones(n, w)), w)
    out = _lib.krylov_solve("bicgstab", w, A, M, b, tol_rel=1e-25)
    assert out["status"] == "OK"


def test_withhold_rejects_bad_rows():
    A_t = inputs.convdiff2d(8, pe=1.0)
    M = _lib.ILU0(_lib.Matrix.from_tuple(A_t), "fp64")
    for bad in (-2, A_t[0]):
        with pytest.raises(_lib.MpkError) as e:
            M.test_withhold(bad)
        assert e.value.status == "INVALID_ARG"
