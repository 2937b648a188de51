"""The seeded input generators against the recipes they state (the stand-ins for the paper's
SuiteSparse matrices and its manufactured solutions, Sec. 4).  CPU only; the generators hold
none of the method's arithmetic, so these checks are of the inputs, not of the solver."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2504_14498_gb300 import inputs


def _dense(A):
    n, rp, ci, v = A
    c = len(v) // len(ci)
    D = np.zeros((n, n), dtype=complex if c == 2 else float)
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            D[i, ci[p]] = v[2 * p] + 1j * v[2 * p + 1] if c == 2 else v[p]
    return D


def _check_csr(A):
    n, rp, ci, v = A
    assert rp[0] == 0 and rp[-1] == len(ci) and np.all(np.diff(rp) >= 1)
    for i in range(n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and i in row  # sorted, diagonal stored


def test_convdiff2d_config_rows():
    """64 x 64, cell Peclet 10 per component, first-order upwind, scaled by h^2: N = 4096,
    nnz = 20,224; interior rows diag 44, west and south -21, east and north -1."""
    A = inputs.convdiff2d(64, pe=10.0)
    n, rp, ci, v = A
    assert n == 4096 and len(ci) == 20224
    _check_csr(A)
    i = 30 * 64 + 30
    row = dict(zip(ci[rp[i]:rp[i + 1]], v[rp[i]:rp[i + 1]]))
    assert row == {i - 64: -21.0, i - 1: -21.0, i: 44.0, i + 1: -1.0, i + 64: -1.0}


def test_convdiff3d_recipe():
    """7-point upwind on m^3 (nnz = 7 m^3 - 6 m^2: 14,581,760 at m = 128), log-normal face
    diffusivities (harmonic means), one global Peclet number in U(1, 50); interior rows conserve
    (row sum 0) and are weakly diagonally dominant; the matrix minus its transpose (convection
    only: the diffusion part is symmetric) is nonzero on exactly the 6 neighbours."""
    assert 7 * 128 ** 3 - 6 * 128 ** 2 == 14581760
    m = 9
    A, meta = inputs.convdiff3d(m)
    n, rp, ci, v = A
    assert n == m ** 3 and len(ci) == 7 * m ** 3 - 6 * m ** 2
    assert 1.0 <= meta["pe"] <= 50.0
    _check_csr(A)
    D = _dense(A)
    for i in (m * m * 4 + m * 4 + 4, m * m * 2 + m * 5 + 3):  # interior cells
        off = D[i].copy()
        off[i] = 0.0
        assert abs(D[i].sum()) <= 1e-12 * D[i, i]
        assert D[i, i] >= np.abs(off).sum() * (1 - 1e-12)
        skew = D[i] - D[:, i]
        assert set(np.nonzero(np.abs(skew) > 1e-12)[0]) == {i - m * m, i - m, i - 1, i + 1, i + m, i + m * m}


def test_helmholtz2d_recipe():
    """h^2 (-Lap - k^2 (1 - 0.5 i)) on m x m, h = 1/(m + 1): nnz = 5 m^2 - 4 m (5,238,784 at
    m = 1024), diagonal 4 - (kh)^2 + 0.5 (kh)^2 i, couplings -1; with k = 20 pi at m = 1024,
    (kh)^2 = 3.7576e-3 and the real part is indefinite."""
    assert 5 * 1024 ** 2 - 4 * 1024 == 5238784
    m, k = 16, 20 * math.pi * 16 / 1024
    A = inputs.helmholtz2d(m, k=k)
    n, rp, ci, v = A
    assert len(ci) == 5 * m * m - 4 * m
    _check_csr(A)
    D = _dense(A)
    kh2 = (k / (m + 1)) ** 2
    assert np.allclose(np.diag(D), 4 - kh2 + 0.5j * kh2, rtol=0, atol=1e-15)
    off = D - np.diag(np.diag(D))
    assert set(np.unique(off[off != 0])) == {-1.0}
    assert abs((20 * math.pi / 1025) ** 2 - 3.7576e-3) < 5e-7


def test_random_sparse_recipe():
    """Entries per row in [kmin, kmax] with the diagonal, distinct columns, diagonal = sum |off|
    (1 + U(0, 0.2)), times 0.6 on the weakened rows (5 %)."""
    A = inputs.random_sparse(400, 3, 40, seed=9)
    n, rp, ci, v = A
    _check_csr(A)
    k = np.diff(rp)
    assert k.min() >= 3 and k.max() <= 40
    ratios = []
    for i in range(n):
        row = v[rp[i]:rp[i + 1]]
        d = row[ci[rp[i]:rp[i + 1]] == i][0]
        ratios.append(d / (np.abs(row).sum() - abs(d)))
    ratios = np.array(ratios)
    strong = (ratios >= 1.0) & (ratios <= 1.2)
    weak = (ratios >= 0.6) & (ratios <= 0.72)
    assert np.all(strong | weak) and 0 < weak.sum() < 0.15 * n


def test_block_diagonal_keeps_systems_apart():
    sys_ = [inputs.random_system(50 + 7 * s, 100 + s, 3, 9) for s in range(4)]
    B, roff = inputs.block_diagonal(sys_)
    n, rp, ci, v = B
    assert n == roff[-1] and len(ci) == sum(len(S[2]) for S in sys_)
    for s in range(4):
        for i in range(roff[s], roff[s + 1]):
            row = ci[rp[i]:rp[i + 1]]
            assert row.min() >= roff[s] and row.max() < roff[s + 1]


@pytest.mark.parametrize("w", [2, 4])
def test_paper_exact_solutions(w):
    """Sec. 4's x = sqrt(2) [1..n] and x = sqrt(2 + 3i) [1..n], each entry the greedy
    w-component rounding of a 100-digit value: (x_k / k)^2 reproduces 2 (and 2 + 3i) to the
    format's precision, and the components are nonoverlapping."""
    n = 7
    tol = Fraction(2) ** (-100 if w == 2 else -195)
    x = inputs.paper_xstar(n, w).reshape(n, w)
    for k in range(1, n + 1):
        r = sum(Fraction(c) for c in x[k - 1]) / k
        assert abs(r * r - 2) <= 2 * tol
        for j in range(w - 1):
            assert abs(x[k - 1, j + 1]) <= abs(x[k - 1, j]) * 2.0 ** -52
    z = inputs.paper_xstar(n, w, complex_=True).reshape(n, 2, w)
    for k in range(1, n + 1):
        a = sum(Fraction(c) for c in z[k - 1, 0]) / k
        b = sum(Fraction(c) for c in z[k - 1, 1]) / k
        assert abs(a * a - b * b - 2) <= 8 * tol and abs(2 * a * b - 3) <= 8 * tol
