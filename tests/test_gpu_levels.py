"""The level structure the library builds for the substitutions and the ILU(0) kernels against
its definition, computed here row by row on the CPU: a row's level is 0 without dependencies in
the triangle, else 1 + the largest level of the rows it depends on (the columns left of the
diagonal for L~, right of it for U~).  Any valid schedule gives the same results, so only this
test sees a wrong level (a deadlock-free but longer order, or a missed dependency)."""
import numpy as np
import pytest

from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu


def _levels(A, lower):
    n, rp, ci, _ = A
    d = np.zeros(n, dtype=np.int64)
    rows = range(n) if lower else range(n - 1, -1, -1)
    for i in rows:
        cols = ci[rp[i]:rp[i + 1]]
        deps = cols[cols < i] if lower else cols[cols > i]
        d[i] = 1 + d[deps].max() if len(deps) else 0
    return d


def _batch():
    sys_ = [inputs.random_system(300 + 41 * k, 700 + k, 3, 14) for k in range(6)]
    B, _ = inputs.block_diagonal(sys_)
    return (B[0], B[1].astype(np.int32), B[2], B[3])


MATS = {
    "convdiff2d": lambda: (inputs.convdiff2d(41, pe=10.0), 1),
    "convdiff3d": lambda: (inputs.convdiff3d(13)[0], 1),
    "random": lambda: (inputs.random_sparse(2000, 3, 20, seed=31), 1),
    "batch": lambda: (_batch(), 1),
    "chain": lambda: (inputs.tridiag(3000, -1.0, 4.0, -1.0), 1),
    "helmholtz": lambda: (inputs.helmholtz2d(29, k=15.0), 2),
}


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "mp2", "mp4"])
def test_levels_match_definition(mat, prec):
    """Every way of building a handle: the binary64 / binary32 / bfloat16 factorisations and the
    multi-component one (mpk_ilu0_factor_mp with w = 2 and 4)."""
    A_t, c = MATS[mat]()
    A = _lib.Matrix.from_tuple(A_t, is_complex=(c == 2))
    M = _lib.ILU0(A, "mp", int(prec[2])) if prec.startswith("mp") else _lib.ILU0(A, prec)
    for tri, lower in ((0, True), (1, False)):
        nl, depth = M.levels(tri)
        ref = _levels(A_t, lower)
        assert np.array_equal(depth.cpu().numpy(), ref), (mat, tri)
        assert nl == ref.max() + 1
    if mat == "convdiff2d":
        assert M.levels(0)[0] == M.levels(1)[0] == 2 * 41 - 1
    if mat == "convdiff3d":
        assert M.levels(0)[0] == 3 * 13 - 2
    if mat == "chain":
        assert M.levels(0)[0] == 3000
