"""Final accuracy against the manufactured solution x* = ones (the error bars of the workload
statement: relative error <= 1e-28 with DD vectors and <= 1e-60 with QD vectors on a
well-conditioned system), with every factor precision: the binary32 / bfloat16 factors win the
accuracy back through the multi-component iteration.  Runs within the stated bars of the
oracle's (tests/_bars.py)."""
import numpy as np
import pytest
import torch

import _bars
import oracle
from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def _relerr(x, w):
    X = np.asarray(x).reshape(-1, w)
    ones = np.zeros_like(X)
    ones[:, 0] = 1.0
    e = _bars.mp_diff(X, ones, w)
    return float(np.linalg.norm(e) / np.sqrt(X.shape[0]))


@pytest.mark.parametrize("w,tol,bar", [(2, 1e-29, 1e-28), (4, 1e-61, 1e-60)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_final_error_on_config_1(w, tol, bar, prec):
    A_t = inputs.convdiff2d(64, pe=10.0)
    n = A_t[0]
    A = _lib.Matrix.from_tuple(A_t)
    b = oracle.spmv(A_t, inputs.ones(n, w), w)
    out = _lib.krylov_solve("bicgstab", w, A, _lib.ILU0(A, prec), torch.as_tensor(b, device="cuda"), tol_rel=tol,
                            maxit=400)
    x = out["x"].cpu().numpy()
    ref = oracle.krylov("bicgstab", A_t, b, w, ilu=prec, tol_rel=tol, maxit=400)
    assert out["status"] == ref["status"] == "OK"
    _bars.check_solve(out, ref, prec, w, tol)
    assert _relerr(x, w) <= bar, _relerr(x, w)
    assert _relerr(ref["x"], w) <= bar, _relerr(ref["x"], w)
