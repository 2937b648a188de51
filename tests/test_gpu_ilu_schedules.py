"""Both schedules of the ILU(0) kernels against the oracle: the level-synchronous one (the rows of
a level dealt over a cooperative grid, grid barriers between levels) and the dataflow over chunk
flags, each forced through MPK_ILU_SCHEDULE (without it the library picks one by the width of the
levels).  Both must return Algorithm 1's factor bit for bit
for every precision, real and complex, on shallow and wide level structures (a batch of
block-diagonal systems), deep ones (a tridiagonal chain: one row per level) and matrices whose
pivot is zero."""
import numpy as np
import pytest

import oracle
from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def _batch():
    sys_ = [inputs.random_system(200 + 37 * k, 900 + k, 3, 12) for k in range(9)]
    B_t, _ = inputs.block_diagonal(sys_)
    return (B_t[0], B_t[1].astype(np.int32), B_t[2], B_t[3])


MATS = {
    "convdiff2d": lambda: (inputs.convdiff2d(41, pe=10.0), 1),
    "convdiff3d": lambda: (inputs.convdiff3d(19)[0], 1),
    "random": lambda: (inputs.random_sparse(2500, 3, 20, seed=14), 1),
    "tridiag_chain": lambda: (inputs.tridiag(3000, -1.0, 4.0, -2.0), 1),
    "batch": lambda: (_batch(), 1),
    "helmholtz": lambda: (inputs.helmholtz2d(31, k=15.0), 2),
}


@pytest.fixture(params=["levels", "dataflow"])
def ilu_schedule(request, monkeypatch):
    monkeypatch.setenv("MPK_ILU_SCHEDULE", request.param)
    return request.param


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "mp1", "mp2"])
def test_factor_matches_oracle(ilu_schedule, mat, prec):
    A_t, c = MATS[mat]()
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    if prec.startswith("mp"):
        w = int(prec[2:])
        M = _lib.ILU0(A, "mp", w)
        st, ref, _ = oracle.ilu0(A_t, "mp", c, w)
    else:
        M = _lib.ILU0(A, prec)
        st, ref, _ = oracle.ilu0(A_t, prec, c)
    assert st == 0
    got = M.values().cpu().numpy()
    assert np.array_equal(got, ref), (mat, prec, np.max(np.abs(got - ref)))
    M.close()


def test_zero_pivot_row_reported(ilu_schedule):
    """a_11 - a_10 a_01 / a_00 = 0 in row 1 of a 5 x 5 tridiagonal band: the factorisation stops
    with MPK_ZERO_PIVOT and fail_row 1 under either schedule."""
    A_t = inputs.tridiag(5, 1.0, 1.0, 1.0)
    with pytest.raises(_lib.MpkError) as e:
        _lib.ILU0(_lib.Matrix.from_tuple(A_t), "fp64")
    assert e.value.status == "ZERO_PIVOT"
    st, _, fr = oracle.ilu0(A_t, "fp64")
    assert st == 3 and fr == 1
