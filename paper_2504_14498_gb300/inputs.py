"""Seeded synthetic inputs shaped like the workloads of the paper and of its GPU-scale configs.

This module only builds matrices and right-hand-side ingredients (exact solutions, random
vectors).  It holds none of the method's arithmetic: b = A x* is computed by whichever side
(the CUDA path or the CPU oracle) consumes the inputs.

Matrices are CSR with int32 row pointers / column indices (columns strictly ascending in each
row, diagonal always stored) and binary64 values; complex values are interleaved (re, im).
A matrix is returned as the tuple (n, row_ptr, col, val) plus a flag for complex.

Recipes (stand-ins for the SuiteSparse matrices mcfe/mpfe and dwg961b of Sec. 4, which are not
available here):
  convdiff2d  -k Lap(u) + v.grad(u) on the unit square, Dirichlet boundary eliminated, 5-point
              first-order upwind, scaled by h^2, h = 1/(m+1), natural (x-fastest) ordering.
              Cell Peclet Pe_d = |v_d| h / (2 k) per axis, so the row is
              diag 4 + 2Pe_x + 2Pe_y, upwind neighbours -1 - 2Pe_d, downwind -1.
  convdiff3d  same in 3-D with a cell-wise log-normal diffusivity k = exp(sigma g), g ~ N(0,1),
              face diffusivity = harmonic mean of the two cells (the cell's own value at a
              boundary face), velocity direction (1, 0.5, 0.25) normalised, one global cell
              Peclet number Pe ~ U(pe_lo, pe_hi) per seeded instance measured against k = 1:
              h v_d = 2 Pe vhat_d.  7-point, natural ordering.
  helmholtz2d h^2 (-Lap - k^2 (1 - 0.5 i)) on the unit square, 5-point, Dirichlet eliminated.
  random_sparse  n x n, K ~ U{kmin..kmax} entries per row (diagonal included) at distinct
              uniform random columns, off-diagonals N(0,1), diagonal = (sum |off|) (1 + U(0, 0.2)),
              a fraction of rows with the diagonal weakened by a factor.
"""
import math
from decimal import Decimal, getcontext

import numpy as np

SEED_BASE = 2504_14498


def _csr_from_rows(n, cols, vals):
    """cols/vals: (n, k) arrays with -1 marking absent entries; columns ascending per row."""
    mask = cols >= 0
    counts = mask.sum(axis=1)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    ci = cols[mask].astype(np.int32)
    if vals.ndim == 3:  # complex: (n, k, 2)
        va = vals[mask].reshape(-1)
    else:
        va = vals[mask]
    return rp.astype(np.int32), ci, np.ascontiguousarray(va, dtype=np.float64)


def convdiff2d(m=64, pe=10.0, kappa=1.0, velocity=(1.0, 1.0)):
    """Config 'plain method, small': 5-point upwind convection-diffusion on an m x m grid."""
    n = m * m
    vx, vy = velocity
    vn = math.hypot(vx, vy)
    # cell Peclet pe per component along the flow direction (1,1): h v_d / (2 kappa) = pe
    pex = pe * abs(vx) / max(abs(vx), abs(vy)) if vn > 0 else 0.0
    pey = pe * abs(vy) / max(abs(vx), abs(vy)) if vn > 0 else 0.0
    idx = np.arange(n)
    ix, iy = idx % m, idx // m
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5))
    # order: south (i-m), west (i-1), centre, east (i+1), north (i+m)
    up_x = -kappa - 2 * kappa * pex if vx >= 0 else -kappa
    dn_x = -kappa if vx >= 0 else -kappa - 2 * kappa * pex
    up_y = -kappa - 2 * kappa * pey if vy >= 0 else -kappa
    dn_y = -kappa if vy >= 0 else -kappa - 2 * kappa * pey
    diag = 4 * kappa + 2 * kappa * pex + 2 * kappa * pey
    s = iy > 0
    cols[s, 0] = idx[s] - m; vals[s, 0] = up_y
    w_ = ix > 0
    cols[w_, 1] = idx[w_] - 1; vals[w_, 1] = up_x
    cols[:, 2] = idx; vals[:, 2] = diag
    e = ix < m - 1
    cols[e, 3] = idx[e] + 1; vals[e, 3] = dn_x
    nn = iy < m - 1
    cols[nn, 4] = idx[nn] + m; vals[nn, 4] = dn_y
    rp, ci, va = _csr_from_rows(n, cols, vals)
    return (n, rp, ci, va)


def convdiff3d(m=128, sigma=1.0, pe_range=(1.0, 50.0), direction=(1.0, 0.5, 0.25), seed=SEED_BASE + 1):
    """Config 'precision': 7-point upwind convection-diffusion with log-normal diffusivity."""
    rng = np.random.default_rng(seed)
    n = m ** 3
    kap = np.exp(sigma * rng.standard_normal(n))
    pe = float(rng.uniform(*pe_range))
    d = np.asarray(direction, dtype=np.float64)
    vh = d / np.linalg.norm(d)
    hv = 2.0 * pe * vh  # h * v_d, measured against kappa = 1
    idx = np.arange(n)
    ix, iy, iz = idx % m, (idx // m) % m, idx // (m * m)
    strides = (1, m, m * m)
    coords = (ix, iy, iz)
    cols = np.full((n, 7), -1, dtype=np.int64)
    vals = np.zeros((n, 7))
    diag = np.zeros(n)
    # slots: 0: -m^2, 1: -m, 2: -1, 3: centre, 4: +1, 5: +m, 6: +m^2
    for axis, (slot_lo, slot_hi) in enumerate(((2, 4), (1, 5), (0, 6))):
        st, c = strides[axis], coords[axis]
        has_lo, has_hi = c > 0, c < m - 1
        k_lo = kap.copy()
        k_lo[has_lo] = 2.0 / (1.0 / kap[has_lo] + 1.0 / kap[idx[has_lo] - st])
        k_hi = kap.copy()
        k_hi[has_hi] = 2.0 / (1.0 / kap[has_hi] + 1.0 / kap[idx[has_hi] + st])
        diag += k_lo + k_hi + hv[axis]
        cols[has_lo, slot_lo] = idx[has_lo] - st
        vals[has_lo, slot_lo] = -k_lo[has_lo] - hv[axis]
        cols[has_hi, slot_hi] = idx[has_hi] + st
        vals[has_hi, slot_hi] = -k_hi[has_hi]
    cols[:, 3] = idx
    vals[:, 3] = diag
    rp, ci, va = _csr_from_rows(n, cols, vals)
    return (n, rp, ci, va), {"pe": pe, "sigma": sigma, "m": m}


def helmholtz2d(m=1024, k=20 * math.pi, damping=0.5):
    """Config 'complex': shifted-Laplacian Helmholtz, h^2(-Lap - k^2 (1 - i damping))."""
    n = m * m
    h = 1.0 / (m + 1)
    kh2 = (k * h) ** 2
    idx = np.arange(n)
    ix, iy = idx % m, idx // m
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5, 2))
    s = iy > 0
    cols[s, 0] = idx[s] - m; vals[s, 0, 0] = -1.0
    w_ = ix > 0
    cols[w_, 1] = idx[w_] - 1; vals[w_, 1, 0] = -1.0
    cols[:, 2] = idx; vals[:, 2, 0] = 4.0 - kh2; vals[:, 2, 1] = kh2 * damping
    e = ix < m - 1
    cols[e, 3] = idx[e] + 1; vals[e, 3, 0] = -1.0
    nn = iy < m - 1
    cols[nn, 4] = idx[nn] + m; vals[nn, 4, 0] = -1.0
    rp, ci, va = _csr_from_rows(n, cols, vals)
    return (n, rp, ci, va)


def magnetic_laplacian2d(m, seed=SEED_BASE + 11, shift=-0.5, flux=1.0):
    """Hermitian test system: the 5-point Laplacian of a charged particle in a random magnetic
    field (a gauge Laplacian), h^2-scaled: diagonal 4 + shift, edge (i, j) couples with
    -exp(i theta_ij) and its mirror with the exact conjugate -exp(-i theta_ij); theta ~
    U(-pi flux, pi flux) per edge, seeded.  A = A^H exactly (the imaginary parts of mirrors are
    exact negations); the random gauge lifts the spectrum's lower edge above the shifted 0."""
    rng = np.random.default_rng(seed)
    n = m * m
    idx = np.arange(n)
    ix, iy = idx % m, idx // m
    th_e = rng.uniform(-math.pi * flux, math.pi * flux, size=n)  # edge to the east neighbour
    th_n = rng.uniform(-math.pi * flux, math.pi * flux, size=n)  # edge to the north neighbour
    ce, se = -np.cos(th_e), -np.sin(th_e)
    cn, sn = -np.cos(th_n), -np.sin(th_n)
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5, 2))
    s = iy > 0  # south neighbour: mirror of its north edge
    cols[s, 0] = idx[s] - m; vals[s, 0, 0] = cn[idx[s] - m]; vals[s, 0, 1] = -sn[idx[s] - m]
    w_ = ix > 0  # west neighbour: mirror of its east edge
    cols[w_, 1] = idx[w_] - 1; vals[w_, 1, 0] = ce[idx[w_] - 1]; vals[w_, 1, 1] = -se[idx[w_] - 1]
    cols[:, 2] = idx; vals[:, 2, 0] = 4.0 + shift
    e = ix < m - 1
    cols[e, 3] = idx[e] + 1; vals[e, 3, 0] = ce[idx[e]]; vals[e, 3, 1] = se[idx[e]]
    nn = iy < m - 1
    cols[nn, 4] = idx[nn] + m; vals[nn, 4, 0] = cn[idx[nn]]; vals[nn, 4, 1] = sn[idx[nn]]
    rp, ci, va = _csr_from_rows(n, cols, vals)
    return (n, rp, ci, va)


def scaled_random_sparse(n=765, k=32, span=5.0, weak_frac=0.5, weak_factor=0.5, seed=SEED_BASE + 21):
    """Stand-in for the paper's real test matrix (Sec. 4, Table 1: n = 765, about 32 stored entries
    per row; without a preconditioner no method reaches 1e-13 within 3n iterations in DD, TD or QD,
    while ILU(0) needs about ten): a nonsymmetric random sparse system with k entries per row and
    weakened diagonal dominance (random_sparse), its rows and columns scaled independently by
    10^U(-span, span).  ILU(0) is unaffected by the scaling (the factors scale with it); the
    unpreconditioned iteration is not."""
    n_, rp, ci, val = random_sparse(n, k, k, weak_frac=weak_frac, weak_factor=weak_factor, seed=seed)
    rng = np.random.default_rng(seed + 1)
    dr = 10.0 ** rng.uniform(-span, span, n)
    dc = 10.0 ** rng.uniform(-span, span, n)
    rows = np.repeat(np.arange(n), np.diff(rp))
    return (n, rp, ci, val * dr[rows] * dc[ci])


def scaled_helmholtz2d(m=31, k=28.0, damping=0.02, span=4.0, seed=SEED_BASE + 22):
    """Stand-in for the paper's complex test matrix (Sec. 4, Table 2: n = 961, complex symmetric;
    without a preconditioner no method converges within 3n iterations, with ILU(0) hundreds to
    about two thousand iterations): the shifted-Laplacian Helmholtz matrix on an m x m grid with a
    small damping (strongly indefinite), scaled symmetrically, D A D with D = diag(10^U(-span,
    span)), which keeps it complex symmetric."""
    n, rp, ci, val = helmholtz2d(m, k=k, damping=damping)
    rng = np.random.default_rng(seed)
    d = 10.0 ** rng.uniform(-span, span, n)
    rows = np.repeat(np.arange(n), np.diff(rp))
    f = d[rows] * d[ci]
    v = val.copy()
    v[0::2] *= f
    v[1::2] *= f
    return (n, rp, ci, v)


def random_sparse(n, kmin=5, kmax=40, weak_frac=0.05, weak_factor=0.6, seed=SEED_BASE + 3, complex_=False):
    """Nonsymmetric random sparse system (diagonally dominant except the weakened rows)."""
    rng = np.random.default_rng(seed)
    kmax = min(kmax, n)
    kmin = min(kmin, kmax)
    k = rng.integers(kmin, kmax + 1, size=n)
    rows_c, rows_v = [], []
    for i in range(n):
        others = rng.choice(n - 1, size=k[i] - 1, replace=False)
        others = others + (others >= i)
        c = np.sort(np.concatenate([others, [i]]))
        if complex_:
            v = rng.standard_normal((k[i], 2))
        else:
            v = rng.standard_normal(k[i])
        rows_c.append(c)
        rows_v.append(v)
    weak = rng.random(n) < weak_frac
    grow = rng.uniform(0.0, 0.2, size=n)
    rp = np.zeros(n + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(c) for c in rows_c])
    ci = np.concatenate(rows_c).astype(np.int32)
    vals = []
    for i in range(n):
        c, v = rows_c[i], rows_v[i]
        d = int(np.nonzero(c == i)[0][0])
        if complex_:
            off = np.abs(v[:, 0] + 1j * v[:, 1])
            s = off.sum() - off[d]
            v[d] = [s * (1 + grow[i]) * (weak_factor if weak[i] else 1.0), 0.0]
        else:
            s = np.abs(v).sum() - abs(v[d])
            v[d] = s * (1 + grow[i]) * (weak_factor if weak[i] else 1.0)
        vals.append(v.reshape(-1))
    return (n, rp, ci, np.concatenate(vals).astype(np.float64))


def tridiag(n, lo, di, up):
    """Tridiagonal matrix with constant (or per-row array) diagonals."""
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (n,))
    di = np.broadcast_to(np.asarray(di, dtype=np.float64), (n,))
    up = np.broadcast_to(np.asarray(up, dtype=np.float64), (n,))
    idx = np.arange(n)
    cols = np.full((n, 3), -1, dtype=np.int64)
    vals = np.zeros((n, 3))
    cols[1:, 0] = idx[1:] - 1; vals[1:, 0] = lo[1:]
    cols[:, 1] = idx; vals[:, 1] = di
    cols[:-1, 2] = idx[:-1] + 1; vals[:-1, 2] = up[:-1]
    rp, ci, va = _csr_from_rows(n, cols, vals)
    return (n, rp, ci, va)


def ones(n, w, c=1):
    """x* = ones as an n-vector of w-component numbers (c = 2: real part 1, imaginary 0)."""
    x = np.zeros((n, c, w))
    x[:, 0, 0] = 1.0
    return x.reshape(-1)


def _split_decimal(d, w):
    comps = []
    for _ in range(w):
        f = float(d)
        comps.append(f)
        d = d - Decimal(f)
    return comps


def paper_xstar(n, w, complex_=False):
    """Exact solution of Sec. 4: x = sqrt(2) [1..n] (real) or sqrt(2 + 3i) [1..n] (complex),
    each entry rounded greedily to w binary64 components from a 100-digit decimal value."""
    getcontext().prec = 100
    if not complex_:
        s = Decimal(2).sqrt()
        return np.array([c for k in range(1, n + 1) for c in _split_decimal(s * k, w)])
    # principal sqrt(2 + 3i) = a + b i, a = sqrt((|z| + 2)/2), b = sqrt((|z| - 2)/2)
    mod = Decimal(13).sqrt()
    a = ((mod + 2) / 2).sqrt()
    b = ((mod - 2) / 2).sqrt()
    out = []
    for k in range(1, n + 1):
        out += _split_decimal(a * k, w) + _split_decimal(b * k, w)
    return np.array(out)


def random_vector(n, w, c=1, seed=SEED_BASE + 7, scale=1.0):
    """Random vector, leading components N(0, scale^2), lower components a random fraction of
    an ulp so that every component is in use (w > 1)."""
    rng = np.random.default_rng(seed)
    v = np.zeros((n, c, w))
    v[:, :, 0] = scale * rng.standard_normal((n, c))
    for k in range(1, w):
        v[:, :, k] = v[:, :, k - 1] * (2.0 ** -53) * rng.uniform(-0.5, 0.5, size=(n, c))
    return v.reshape(-1)


def normal_rhs(n, w, c=2, seed=SEED_BASE + 3):
    """Right-hand side with N(0, 1) leading components (real and imaginary parts when c = 2) and
    zero lower components: the Helmholtz workload's random b."""
    rng = np.random.default_rng(seed)
    v = np.zeros((n, c, w))
    v[:, :, 0] = rng.standard_normal((n, c))
    return v.reshape(-1)


def random_system(n, seed, kmin=5, kmax=40, weak_frac=0.05, weak_factor=0.6):
    """One system of the batched workload (vectorised recipe of random_sparse): n x n, K ~
    U{kmin..kmax} entries per row including the diagonal, off-diagonal columns distinct and
    uniform among the other n-1, off-diagonals N(0,1), diagonal = (sum |off|)(1 + U(0, 0.2)),
    weakened by weak_factor in a weak_frac share of the rows.  Returns (n, row_ptr, col, val)."""
    rng = np.random.default_rng(seed)
    kmax = min(kmax, n)
    kmin = min(kmin, kmax)
    k = rng.integers(kmin, kmax + 1, size=n)
    rows = np.repeat(np.arange(n, dtype=np.int64), k - 1)
    cols = rng.integers(0, n - 1, size=len(rows), dtype=np.int64)
    cols += cols >= rows
    for _ in range(64):  # redraw duplicated columns of a row until all are distinct
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        rows, cols = rows[order], cols[order]
        dup = np.zeros(len(rows), dtype=bool)
        dup[1:] = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        nd = int(dup.sum())
        if nd == 0:
            break
        c = rng.integers(0, n - 1, size=nd, dtype=np.int64)
        cols[dup] = c + (c >= rows[dup])
    off = rng.standard_normal(len(rows))
    weak = rng.random(n) < weak_frac
    grow = rng.uniform(0.0, 0.2, size=n)
    rsum = np.bincount(rows, weights=np.abs(off), minlength=n)
    diag = rsum * (1.0 + grow) * np.where(weak, weak_factor, 1.0)
    rows_all = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    cols_all = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    vals_all = np.concatenate([off, diag])
    order = np.argsort(rows_all * n + cols_all, kind="stable")
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(k, out=rp[1:])
    return (n, rp.astype(np.int32), cols_all[order].astype(np.int32), vals_all[order].astype(np.float64))


def batch_sizes(nsys=512, nmin=1000, nmax=200000, seed=SEED_BASE + 4):
    """System sizes of the batched workload: N log-uniform in [nmin, nmax]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=nsys)).astype(np.int64)


def batch_system(s, sizes, seed=SEED_BASE + 4000):
    """System s of the batch (its own seed, so any one system can be rebuilt alone)."""
    return random_system(int(sizes[s]), seed + int(s))


def batch_xstar(n, w, seed):
    """Exact solution of one batch system: leading components U(-1, 1)."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n, w))
    x[:, 0] = rng.uniform(-1.0, 1.0, size=n)
    return x.reshape(-1)


def block_diagonal(systems):
    """Concatenate CSR systems into one block-diagonal CSR (global column indices) and the row
    offsets of the systems (int64 for the total entry count; the library takes int32)."""
    ns = np.array([A[0] for A in systems], dtype=np.int64)
    roff = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(ns, out=roff[1:])
    nnzs = np.array([len(A[2]) for A in systems], dtype=np.int64)
    eoff = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(nnzs, out=eoff[1:])
    rp = np.empty(int(roff[-1]) + 1, dtype=np.int64)
    ci = np.empty(int(eoff[-1]), dtype=np.int32)
    val = np.empty(int(eoff[-1]) * (len(systems[0][3]) // max(1, len(systems[0][2]))), dtype=np.float64)
    c = len(systems[0][3]) // max(1, len(systems[0][2]))
    for s, A in enumerate(systems):
        n, r, cc, v = A
        rp[roff[s]:roff[s] + n] = r[:-1].astype(np.int64) + eoff[s]
        ci[eoff[s]:eoff[s + 1]] = cc + roff[s]
        val[eoff[s] * c:eoff[s + 1] * c] = v
    rp[-1] = eoff[-1]
    return (int(roff[-1]), rp, ci, val), roff


_PATTERN_2D = {}


def _pattern2d(m):
    """5-point pattern of an m x m grid (natural ordering) and, per slot (-m, -1, centre, +1, +m),
    the CSR position of each row's entry (-1 where the neighbour does not exist)."""
    if m not in _PATTERN_2D:
        n = m * m
        idx = np.arange(n)
        ix, iy = idx % m, idx // m
        cols = np.full((n, 5), -1, dtype=np.int64)
        cols[iy > 0, 0] = idx[iy > 0] - m
        cols[ix > 0, 1] = idx[ix > 0] - 1
        cols[:, 2] = idx
        cols[ix < m - 1, 3] = idx[ix < m - 1] + 1
        cols[iy < m - 1, 4] = idx[iy < m - 1] + m
        mask = cols >= 0
        rp = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(mask.sum(axis=1), out=rp[1:])
        slotpos = np.full((n, 5), -1, dtype=np.int64)
        slotpos[mask] = np.arange(int(rp[-1]))
        _PATTERN_2D[m] = (rp.astype(np.int32), cols[mask].astype(np.int32), slotpos)
    return _PATTERN_2D[m]


def convdiff2d_random(m, seed, sigma=1.0, pe_range=(1.0, 100.0)):
    """Learned-preconditioner workload: 5-point first-order upwind convection-diffusion on an
    m x m grid with a node-wise log-normal diffusivity k = exp(sigma g), g ~ N(0,1) (face value =
    harmonic mean of the two nodes, the node's own value at a boundary face), a random flow
    direction theta ~ U(0, 2 pi) and one cell Peclet number Pe ~ U(pe_lo, pe_hi) measured against
    k = 1 (h v_d = 2 Pe (cos theta, sin theta)_d); upwind side chosen by the sign of v_d; scaled by
    h^2, natural ordering.  Returns (n, row_ptr, col, val)."""
    rng = np.random.default_rng(seed)
    n = m * m
    kap = np.exp(sigma * rng.standard_normal(n))
    theta = float(rng.uniform(0.0, 2.0 * math.pi))
    pe = float(rng.uniform(*pe_range))
    hv = (2.0 * pe * math.cos(theta), 2.0 * pe * math.sin(theta))
    rp, ci, slotpos = _pattern2d(m)
    kg = kap.reshape(m, m)  # [y, x]
    val = np.zeros(len(ci))
    diag = np.zeros((m, m))
    # axis 0: x (stride 1, slots 1 / 3), axis 1: y (stride m, slots 0 / 4)
    for axis, (slot_lo, slot_hi) in enumerate(((1, 3), (0, 4))):
        k = kg if axis == 0 else kg.T  # k[.., c] runs along the axis
        face = 2.0 / (1.0 / k[:, 1:] + 1.0 / k[:, :-1])  # between c and c+1
        k_lo = k.copy()
        k_lo[:, 1:] = face
        k_hi = k.copy()
        k_hi[:, :-1] = face
        if axis == 1:
            k_lo, k_hi = k_lo.T, k_hi.T
        up_lo, up_hi = max(hv[axis], 0.0), max(-hv[axis], 0.0)
        diag += k_lo + k_hi + up_lo + up_hi
        lo = slotpos[:, slot_lo]
        hi = slotpos[:, slot_hi]
        klo, khi = k_lo.reshape(-1), k_hi.reshape(-1)
        val[lo[lo >= 0]] = -klo[lo >= 0] - up_lo
        val[hi[hi >= 0]] = -khi[hi >= 0] - up_hi
    val[slotpos[:, 2]] = diag.reshape(-1)
    return (n, rp.copy(), ci.copy(), val)


def probe_vectors(n, k, seed):
    """k random probe vectors with N(0,1) entries (binary32), n x k row-major: the learned
    preconditioner's training losses are estimated over such vectors."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, k)).astype(np.float32)


def smooth_probes(m, nsys, k, seed, modes=4):
    """k smooth probe vectors per m x m grid system, for nsys stacked systems (binary32,
    (nsys m^2) x k row-major): sums of the grid's lowest sine modes sin(a pi x) sin(b pi y),
    a, b = 1..modes, with N(0,1) / (a b) coefficients."""
    rng = np.random.default_rng(seed)
    x = (np.arange(m) + 1.0) / (m + 1.0)
    S = np.stack([np.sin(a * np.pi * x) for a in range(1, modes + 1)])  # [modes, m]
    out = np.empty((nsys, m * m, k), dtype=np.float32)
    w = 1.0 / np.outer(np.arange(1, modes + 1), np.arange(1, modes + 1))
    for s_ in range(nsys):
        for c in range(k):
            C = rng.standard_normal((modes, modes)) * w  # C[b, a]: y mode b, x mode a
            out[s_, :, c] = (S.T @ C @ S).reshape(-1)  # [y, x], natural ordering y * m + x
    return out.reshape(nsys * m * m, k)


def convdiff3d_random(m, seed, sigma=1.0, pe_range=(1.0, 50.0), direction=(1.0, 0.5, 0.25)):
    """Training instances of the learned correction for the 3-D workload: the 7-point recipe of
    convdiff3d on an m^3 grid with its own seeded log-normal diffusivity field and Peclet
    number (the same distribution as the 128^3 configuration, other seeds)."""
    A, _ = convdiff3d(m, sigma=sigma, pe_range=pe_range, direction=direction, seed=seed)
    return A


def smooth_probes3d(m, nsys, k, seed, modes=3):
    """k smooth probe vectors per m^3 grid system (binary32, (nsys m^3) x k row-major): sums of
    the lowest sine modes sin(a pi x) sin(b pi y) sin(c pi z), a, b, c = 1..modes, with
    N(0,1) / (a b c) coefficients; natural ordering (x fastest)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(m) + 1.0) / (m + 1.0)
    S = np.stack([np.sin(a * np.pi * x) for a in range(1, modes + 1)])  # [modes, m]
    f = np.arange(1, modes + 1, dtype=np.float64)
    w = 1.0 / (f[:, None, None] * f[None, :, None] * f[None, None, :])  # [c, b, a]
    out = np.empty((nsys, m ** 3, k), dtype=np.float32)
    for s_ in range(nsys):
        for col in range(k):
            C = rng.standard_normal((modes, modes, modes)) * w
            out[s_, :, col] = np.einsum("cba,cz,by,ax->zyx", C, S, S, S).reshape(-1)
    return out.reshape(nsys * m ** 3, k)


def training_probes3d(m, nsys, k, seed):
    """Probe vectors for 3-D training batches: half smooth (smooth_probes3d), half N(0,1)."""
    ks = k // 2
    sm = smooth_probes3d(m, nsys, ks, seed)
    rn = probe_vectors(nsys * m ** 3, k - ks, seed + 1)
    return np.ascontiguousarray(np.concatenate([sm, rn], axis=1), dtype=np.float32)


def training_probes(m, nsys, k, seed):
    """Probe vectors of the learned correction's training: half smooth (smooth_probes), half
    N(0,1) (probe_vectors)."""
    ks = k // 2
    sm = smooth_probes(m, nsys, ks, seed)
    rn = probe_vectors(nsys * m * m, k - ks, seed + 1)
    return np.ascontiguousarray(np.concatenate([sm, rn], axis=1), dtype=np.float32)


GNN_NPARAMS = 12193  # parameter count of the learned correction's network (layout in csrc/gnn.cu)


def gnn_init_params(seed, hidden=32, node_in=4, edge_in=4, layers=3):
    """Seeded initial parameters of the learned-correction network, in its parameter layout
    (encoder W0 [node_in][hidden], b0; per layer Wm [hidden+edge_in][hidden], bm, Wu [2 hidden]
    [hidden], bu; decoder Wd [2 hidden+edge_in][hidden], bd, wo, bo): weights uniform in
    +-1/sqrt(fan_in), biases zero, output layer (wo, bo) zero so that the untrained network's
    output is zero (the plain ILU(0) factor)."""
    H = hidden
    rng = np.random.default_rng(seed)
    P = np.zeros(GNN_NPARAMS, dtype=np.float32)

    def fill(off, fan_in, cnt):
        P[off:off + cnt] = rng.uniform(-1.0, 1.0, cnt) / np.sqrt(fan_in)

    fill(0, node_in, node_in * H)
    base = node_in * H + H
    lsize = (H + edge_in) * H + H + 2 * H * H + H
    for L in range(layers):
        b = base + L * lsize
        fill(b, H + edge_in, (H + edge_in) * H)
        fill(b + (H + edge_in) * H + H, 2 * H, 2 * H * H)
    fill(base + layers * lsize, 2 * H + edge_in, (2 * H + edge_in) * H)
    return P
