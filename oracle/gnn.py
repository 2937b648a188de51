"""Oracle of the learned ILU(0) correction (TEST INFRASTRUCTURE; only tests/ and the smoke check
use it).  Plain numpy in binary64: the graph network's forward pass, the training loss
||(L'U' - A) W||^2 / ||A W||^2 per system, and the gradients by hand-written reverse mode.

The paper has no learned preconditioner; this restates the learned correction of the library
(3 message-passing layers, hidden width 32, binary32 weights, bfloat16 activations) exactly as the
library defines it:
  node input  x_i = (1, sum_{j!=i} |a_ij| / a_ii, sum_j a_ij / a_ii, f_ii / a_ii)
  edge input  e_p = (a_ij / a_ii, a_ji / a_jj (1 on the diagonal, 0 if a_ji is not stored),
                     f_ij / a_ii, sign(j - i))                        p = stored entry (i, j)
  h0_i = bf16(relu(x_i W0 + b0))
  layer: a_i = bf16(sum_{p in row i, j != i} relu([h_j, e_p] Wm + bm)),
         h'_i = bf16(h_i + relu([h_i, a_i] Wu + bu))                  (3 layers)
  o_p = relu([h_i, h_j, e_p] Wd + bd) . wo + bo
  corrected factor f'_p = f_p (1 + 0.5 tanh o_p)
Weight matrices are [in][out]; the parameter vector layout is the library's.  The rounding of a
stored activation to bfloat16 (round to nearest even) is emulated; with round_bf16=False it is
skipped, which makes the forward pass smooth so that finite differences can check the gradients
(the gradient formulas are the same: the rounding is passed through unchanged).

Parity pins: tests/test_oracle_gnn.py (finite differences of the loss with respect to the
parameters and to o; the loss against an explicit dense (L'U' - A) W; o = 0 reproducing ILU(0)).
"""
import numpy as np

H, FN, FE, NL = 32, 4, 4, 3
P_W0, P_B0 = 0, FN * H
L_WM, L_BM = 0, (H + FE) * H
L_WU = L_BM + H
L_BU = L_WU + 2 * H * H
L_SIZE = L_BU + H
P_L0 = P_B0 + H
P_DEC = P_L0 + NL * L_SIZE
D_WD, D_BD = 0, (2 * H + FE) * H
D_WO = D_BD + H
D_BO = D_WO + H
NPARAMS = P_DEC + D_BO + 1


def bf16(x, on=True):
    """Round to bfloat16 (nearest even) through binary32, returned as binary64."""
    if not on:
        return np.asarray(x, dtype=np.float64)
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    d = {"W0": P[P_W0:P_W0 + FN * H].reshape(FN, H), "b0": P[P_B0:P_B0 + H], "layers": []}
    for L in range(NL):
        b = P_L0 + L * L_SIZE
        d["layers"].append({"Wm": P[b + L_WM:b + L_BM].reshape(H + FE, H), "bm": P[b + L_BM:b + L_WU],
                            "Wu": P[b + L_WU:b + L_BU].reshape(2 * H, H), "bu": P[b + L_BU:b + L_SIZE]})
    b = P_DEC
    d["Wd"] = P[b + D_WD:b + D_BD].reshape(2 * H + FE, H)
    d["bd"] = P[b + D_BD:b + D_WO]
    d["wo"] = P[b + D_WO:b + D_BO]
    d["bo"] = P[b + D_BO]
    return d


def _rows(rp):
    n = len(rp) - 1
    return np.repeat(np.arange(n), np.diff(rp))


def diag_positions(A):
    n, rp, ci, _ = A
    rows = _rows(rp)
    d = np.full(n, -1)
    hit = ci == rows
    d[rows[hit]] = np.nonzero(hit)[0]
    return d


def features(A, fac):
    """Node and edge inputs (binary32 values, as the library computes them)."""
    n, rp, ci, a = A
    rows = _rows(rp)
    diag = diag_positions(A)
    aii = a[diag]
    inv = np.where(aii != 0.0, 1.0 / np.where(aii != 0.0, aii, 1.0), 0.0)
    f32 = np.asarray(fac, dtype=np.float32).astype(np.float64)
    pos = {(int(i), int(j)): p for p, (i, j) in enumerate(zip(rows, ci))}
    aji = np.zeros(len(ci))
    for p, (i, j) in enumerate(zip(rows, ci)):
        if i == j:
            aji[p] = 1.0
        else:
            q = pos.get((int(j), int(i)))
            if q is not None:
                ajj = a[diag[j]]
                aji[p] = a[q] / ajj if ajj != 0.0 else 0.0
    sgn = np.sign(rows - ci).astype(np.float64)
    xe = np.stack([a * inv[rows], aji, f32 * inv[rows], sgn], axis=1)
    sabs = np.zeros(n)
    ssum = np.zeros(n)
    for p, (i, j) in enumerate(zip(rows, ci)):  # CSR order, as the library sums
        ssum[i] += a[p]
        if i != j:
            sabs[i] += abs(a[p])
    xn = np.stack([np.ones(n), sabs * np.abs(inv), ssum * inv, f32[diag] * inv], axis=1)
    return xn.astype(np.float32).astype(np.float64), xe.astype(np.float32).astype(np.float64), rows


def forward(P, A, fac, round_bf16=True):
    """Network output o (one value per stored entry) and the cache the backward pass needs."""
    n, rp, ci, a = A
    w = unpack(P)
    xn, xe, rows = features(A, fac)
    off = rows != ci
    h = bf16(np.maximum(xn @ w["W0"] + w["b0"], 0.0), round_bf16)
    hs, as_, pre_m, pre_u = [h], [], [], []
    for lw in w["layers"]:
        pm = np.concatenate([h[ci], xe], axis=1) @ lw["Wm"] + lw["bm"]  # every stored entry
        m = np.where(off[:, None], np.maximum(pm, 0.0), 0.0)
        agg = np.zeros((n, H))
        np.add.at(agg, rows, m)
        agg = bf16(agg, round_bf16)
        q = np.concatenate([h, agg], axis=1) @ lw["Wu"] + lw["bu"]
        h = bf16(h + np.maximum(q, 0.0), round_bf16)
        pre_m.append(pm)
        pre_u.append(q)
        as_.append(agg)
        hs.append(h)
    zin = np.concatenate([h[rows], h[ci], xe], axis=1)
    pd = zin @ w["Wd"] + w["bd"]
    o = np.maximum(pd, 0.0) @ w["wo"] + w["bo"]
    cache = {"xn": xn, "xe": xe, "rows": rows, "off": off, "hs": hs, "as": as_, "pre_m": pre_m,
             "pre_u": pre_u, "zin": zin, "pd": pd}
    return o, cache


def corrected(fac, o):
    return np.asarray(fac, dtype=np.float64) * (1.0 + 0.5 * np.tanh(o))


def loss(A, fac, o, W, sys_rows=None):
    """Training loss and its gradient with respect to o."""
    n, rp, ci, a = A
    rows = _rows(rp)
    W = np.asarray(W, dtype=np.float64).reshape(n, -1)
    fac = np.asarray(fac, dtype=np.float64)
    th = np.tanh(o)
    fp = fac * (1.0 + 0.5 * th)
    low = ci < rows
    upp = ~low
    u = np.zeros_like(W)
    np.add.at(u, rows[upp], fp[upp, None] * W[ci[upp]])
    v = u.copy()
    np.add.at(v, rows[low], fp[low, None] * u[ci[low]])
    aw = np.zeros_like(W)
    np.add.at(aw, rows, a[:, None] * W[ci])
    r = v - aw
    sys_rows = np.array([0, n]) if sys_rows is None else np.asarray(sys_rows)
    nsys = len(sys_rows) - 1
    sid = np.repeat(np.arange(nsys), np.diff(sys_rows))
    R = np.bincount(sid, weights=(r * r).sum(axis=1), minlength=nsys)
    D = np.bincount(sid, weights=(aw * aw).sum(axis=1), minlength=nsys)
    L = float(np.mean(np.where(D > 0, R / np.where(D > 0, D, 1.0), 0.0)))
    coef = np.where(D > 0, 2.0 / (nsys * np.where(D > 0, D, 1.0)), 0.0)[sid]
    gr = coef[:, None] * r
    gfp = np.zeros(len(ci))
    gfp[low] = (gr[rows[low]] * u[ci[low]]).sum(axis=1)
    gu = gr.copy()
    np.add.at(gu, ci[low], fp[low, None] * gr[rows[low]])
    gfp[upp] = (gu[rows[upp]] * W[ci[upp]]).sum(axis=1)
    go = gfp * fac * 0.5 * (1.0 - th * th)
    return L, go


def backward(P, A, cache, go):
    """d loss / d P from d loss / d o (reverse mode through the decoder, layers and encoder)."""
    n, rp, ci, a = A
    w = unpack(P)
    G = np.zeros(NPARAMS)
    rows, xe, off = cache["rows"], cache["xe"], cache["off"]
    pd, zin = cache["pd"], cache["zin"]
    hid = np.maximum(pd, 0.0)
    G[P_DEC + D_WO:P_DEC + D_BO] = hid.T @ go
    G[P_DEC + D_BO] = go.sum()
    gpd = np.where(pd > 0, go[:, None] * w["wo"][None, :], 0.0)
    G[P_DEC + D_WD:P_DEC + D_BD] = (zin.T @ gpd).reshape(-1)
    G[P_DEC + D_BD:P_DEC + D_WO] = gpd.sum(axis=0)
    gz = gpd @ w["Wd"].T
    gh = np.zeros((n, H))
    np.add.at(gh, rows, gz[:, :H])
    np.add.at(gh, ci, gz[:, H:2 * H])
    for L in range(NL - 1, -1, -1):
        lw = w["layers"][L]
        b = P_L0 + L * L_SIZE
        h, agg = cache["hs"][L], cache["as"][L]
        q, pm = cache["pre_u"][L], cache["pre_m"][L]
        gq = np.where(q > 0, gh, 0.0)
        G[b + L_WU:b + L_BU] = (np.concatenate([h, agg], axis=1).T @ gq).reshape(-1)
        G[b + L_BU:b + L_SIZE] = gq.sum(axis=0)
        gin = gq @ lw["Wu"].T
        gh_new = gh + gin[:, :H]
        ga = gin[:, H:]
        gpm = np.where(off[:, None] & (pm > 0), ga[rows], 0.0)
        G[b + L_WM:b + L_BM] = (np.concatenate([h[ci], xe], axis=1).T @ gpm).reshape(-1)
        G[b + L_BM:b + L_WU] = gpm.sum(axis=0)
        np.add.at(gh_new, ci, (gpm @ lw["Wm"].T)[:, :H])
        gh = gh_new
    pre0 = cache["xn"] @ w["W0"] + w["b0"]
    g0 = np.where(pre0 > 0, gh, 0.0)
    G[P_W0:P_W0 + FN * H] = (cache["xn"].T @ g0).reshape(-1)
    G[P_B0:P_B0 + H] = g0.sum(axis=0)
    return G


def adam(P, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    P = P - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return P, m, v


def _tri_mats(A, fp):
    import scipy.sparse as sp

    n, rp, ci, _ = A
    rows = _rows(rp)
    low = ci < rows
    L = sp.csr_matrix((np.concatenate([fp[low], np.ones(n)]),
                       (np.concatenate([rows[low], np.arange(n)]), np.concatenate([ci[low], np.arange(n)]))), shape=(n, n))
    U = sp.csr_matrix((fp[~low], (rows[~low], ci[~low])), shape=(n, n))
    return L, U


def loss_precond(A, fac, o, W, sys_rows=None):
    """Loss of the preconditioned operator, mean_s ||(M'^-1 A W - W)_s||^2 / ||W_s||^2 with
    M' = L'U' from the corrected factor, and its gradient with respect to o (adjoint solves)."""
    from scipy.sparse.linalg import spsolve_triangular
    import scipy.sparse as sp

    n, rp, ci, a = A
    rows = _rows(rp)
    W = np.asarray(W, dtype=np.float64).reshape(n, -1)
    fac = np.asarray(fac, dtype=np.float64)
    th = np.tanh(o)
    fp = fac * (1.0 + 0.5 * th)
    L, U = _tri_mats(A, fp)
    Am = sp.csr_matrix((a, (rows, ci)), shape=(n, n))
    t = spsolve_triangular(L, Am @ W, lower=True, unit_diagonal=True)
    z = spsolve_triangular(U, t, lower=False)
    r = z - W
    sys_rows = np.array([0, n]) if sys_rows is None else np.asarray(sys_rows)
    nsys = len(sys_rows) - 1
    sid = np.repeat(np.arange(nsys), np.diff(sys_rows))
    R = np.bincount(sid, weights=(r * r).sum(axis=1), minlength=nsys)
    D = np.bincount(sid, weights=(W * W).sum(axis=1), minlength=nsys)
    Lval = float(np.mean(np.where(D > 0, R / np.where(D > 0, D, 1.0), 0.0)))
    gz = np.where(D > 0, 2.0 / (nsys * np.where(D > 0, D, 1.0)), 0.0)[sid][:, None] * r
    lam = spsolve_triangular(sp.csr_matrix(U.T), gz, lower=True)
    mu = spsolve_triangular(sp.csr_matrix(L.T), lam, lower=False, unit_diagonal=True)
    low = ci < rows
    gfp = np.where(low, -(mu[rows] * t[ci]).sum(axis=1), -(lam[rows] * z[ci]).sum(axis=1))
    go = gfp * fac * 0.5 * (1.0 - th * th)
    return Lval, go
