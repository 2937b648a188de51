"""Pins of the learned-correction oracle (oracle/gnn.py) to things other than itself:
finite differences of its forward pass and loss (the gradients), an explicit dense evaluation of
the factorisation-error loss, the exactness of ILU(0) on A's pattern when the correction is zero,
the batch loss as the mean of the systems' losses, and closed forms of the Adam step."""
import numpy as np
import pytest

import oracle
from oracle import gnn
from paper_2504_14498_gb300 import inputs


def _case(m=6, seed=5, prec="fp32"):
    A = inputs.convdiff2d_random(m, seed)
    st, fac, _ = oracle.ilu0(A, prec)
    assert st == 0
    if prec == "fp32":
        fac = fac.astype(np.float32).astype(np.float64)
    W = inputs.probe_vectors(A[0], 3, seed + 1).astype(np.float64)
    return A, fac, W


def _params(seed=1):
    P = inputs.gnn_init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    P[gnn.P_DEC + gnn.D_WO:gnn.P_DEC + gnn.D_BO] = rng.uniform(-0.3, 0.3, gnn.H)  # let gradients flow
    P[gnn.P_DEC + gnn.D_BO] = 0.05
    return P


def _loss_of_P(P, A, fac, W):
    o, _ = gnn.forward(P, A, fac, round_bf16=False)
    return gnn.loss(A, fac, o, W)[0]


def test_param_gradient_matches_finite_differences():
    A, fac, W = _case()
    P = _params()
    o, cache = gnn.forward(P, A, fac, round_bf16=False)
    L, go = gnn.loss(A, fac, o, W)
    G = gnn.backward(P, A, cache, go)
    rng = np.random.default_rng(7)
    for _ in range(8):
        d = rng.standard_normal(gnn.NPARAMS)
        eps = 1e-6
        fd = (_loss_of_P(P + eps * d, A, fac, W) - _loss_of_P(P - eps * d, A, fac, W)) / (2 * eps)
        assert abs(fd - G @ d) <= 1e-5 * max(1.0, abs(fd)), (fd, G @ d)
    # per block of parameters too (a transposed or misplaced block fails here)
    for off, cnt in [(gnn.P_W0, gnn.FN * gnn.H), (gnn.P_L0 + gnn.L_WM, 36 * 32), (gnn.P_L0 + gnn.L_WU, 64 * 32),
                     (gnn.P_L0 + 2 * gnn.L_SIZE + gnn.L_BU, 32), (gnn.P_DEC + gnn.D_WD, 68 * 32)]:
        d = np.zeros(gnn.NPARAMS)
        d[off:off + cnt] = rng.standard_normal(cnt)
        eps = 1e-6
        fd = (_loss_of_P(P + eps * d, A, fac, W) - _loss_of_P(P - eps * d, A, fac, W)) / (2 * eps)
        assert abs(fd - G @ d) <= 1e-5 * max(1e-3, abs(fd)), (off, fd, G @ d)


def test_loss_gradient_in_o_matches_finite_differences():
    A, fac, W = _case(seed=9)
    rng = np.random.default_rng(3)
    o = rng.uniform(-1, 1, len(A[2]))
    L, go = gnn.loss(A, fac, o, W)
    for _ in range(6):
        d = rng.standard_normal(len(o))
        eps = 1e-6
        fd = (gnn.loss(A, fac, o + eps * d, W)[0] - gnn.loss(A, fac, o - eps * d, W)[0]) / (2 * eps)
        assert abs(fd - go @ d) <= 1e-6 * max(1.0, abs(fd))


def _dense(A):
    n, rp, ci, v = A
    D = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    D[rows, ci] = v
    return D


def test_loss_equals_dense_factorisation_error():
    A, fac, W = _case(m=5, seed=11)
    n, rp, ci, _ = A
    rng = np.random.default_rng(4)
    o = rng.uniform(-0.5, 0.5, len(ci))
    fp = gnn.corrected(fac, o)
    F = _dense((n, rp, ci, fp))
    Lm = np.tril(F, -1) + np.eye(n)
    Um = np.triu(F)
    E = Lm @ Um - _dense(A)
    ref = np.sum((E @ W) ** 2) / np.sum((_dense(A) @ W) ** 2)
    assert abs(gnn.loss(A, fac, o, W)[0] - ref) <= 1e-12 * ref


def test_zero_correction_is_ilu0_exact_on_pattern():
    A, fac, W = _case(m=7, seed=13, prec="fp64")
    n, rp, ci, _ = A
    P = inputs.gnn_init_params(2)
    o, _ = gnn.forward(P, A, fac)
    assert np.all(o == 0.0)  # zero output layer: the untrained network is the plain factor
    assert np.array_equal(gnn.corrected(fac, o), fac)
    F = _dense((n, rp, ci, fac))
    E = (np.tril(F, -1) + np.eye(n)) @ np.triu(F) - _dense(A)
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.max(np.abs(E[rows, ci])) <= 1e-12 * np.max(np.abs(A[3]))  # ILU(0): exact on the pattern
    assert np.max(np.abs(E)) > 1e-3  # and not exact off it (fill)


def test_batch_loss_is_mean_of_system_losses():
    A1, f1, W1 = _case(m=5, seed=21)
    A2, f2, W2 = _case(m=6, seed=22)
    B, roff = inputs.block_diagonal([A1, A2])
    B = (B[0], B[1].astype(np.int32), B[2], B[3])
    rng = np.random.default_rng(1)
    o1, o2 = rng.uniform(-1, 1, len(A1[2])), rng.uniform(-1, 1, len(A2[2]))
    Lb, _ = gnn.loss(B, np.concatenate([f1, f2]), np.concatenate([o1, o2]), np.concatenate([W1, W2]), roff)
    ref = 0.5 * (gnn.loss(A1, f1, o1, W1)[0] + gnn.loss(A2, f2, o2, W2)[0])
    assert abs(Lb - ref) <= 1e-13 * ref


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 1.0 + 2.0 ** -8 + 2.0 ** -20])
    got = gnn.bf16(x)
    ref = np.array([1.0, 1.0, 1.0 + 4 * 2.0 ** -8, 1.0, -2.5, 1.0 + 2 * 2.0 ** -8])
    assert np.array_equal(got, ref)


def test_precond_loss_gradient_matches_finite_differences():
    A, fac, W = _case(seed=31)
    rng = np.random.default_rng(8)
    o = rng.uniform(-1, 1, len(A[2]))
    L, go = gnn.loss_precond(A, fac, o, W)
    for _ in range(6):
        d = rng.standard_normal(len(o))
        eps = 1e-6
        fd = (gnn.loss_precond(A, fac, o + eps * d, W)[0] - gnn.loss_precond(A, fac, o - eps * d, W)[0]) / (2 * eps)
        assert abs(fd - go @ d) <= 1e-6 * max(1.0, abs(fd))


def test_precond_loss_equals_dense_evaluation():
    A, fac, W = _case(m=5, seed=33)
    n, rp, ci, _ = A
    o = np.random.default_rng(6).uniform(-0.5, 0.5, len(ci))
    F = _dense((n, rp, ci, gnn.corrected(fac, o)))
    Mi = np.linalg.inv((np.tril(F, -1) + np.eye(n)) @ np.triu(F))
    ref = np.sum((Mi @ _dense(A) @ W - W) ** 2) / np.sum(W ** 2)
    assert abs(gnn.loss_precond(A, fac, o, W)[0] - ref) <= 1e-10 * ref
    # exact LU (no fill: tridiagonal) gives M = A and zero loss
    T = inputs.tridiag(9, -1.0, 2.5, -0.7)
    _, ft, _ = oracle.ilu0(T, "fp64")
    assert gnn.loss_precond(T, ft, np.zeros(len(T[2])), inputs.probe_vectors(9, 2, 1))[0] < 1e-28


def test_adam_closed_forms():
    """Adam (Kingma and Ba, 2015) with its bias corrections: under a constant gradient g the
    corrected moments are exactly g and g^2 at every step, so step k leaves P = -k lr g / (|g| +
    eps); the first step of any gradient moves by lr g / (|g| + eps); and when the gradient flips
    to -g at step 2 the corrected moments are -g (1 - b1) / (1 + b1) and g^2."""
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    g = np.array([3.0, -0.5, 1e-3, 2.0])
    P, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for step in range(1, 6):
        P, m, v = gnn.adam(P, g, m, v, lr, step)
        np.testing.assert_allclose(P, -step * lr * g / (np.abs(g) + eps), rtol=1e-12)
    P1, _, _ = gnn.adam(np.ones(4), -g, np.zeros(4), np.zeros(4), lr, 1)
    np.testing.assert_allclose(P1, 1.0 + lr * g / (np.abs(g) + eps), rtol=1e-12)
    P, m, v = gnn.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), lr, 1)
    P, m, v = gnn.adam(P, -g, m, v, lr, 2)
    m_hat = -g * (1 - b1) / (1 + b1)
    step2 = -lr * m_hat / (np.abs(g) + eps)
    np.testing.assert_allclose(P, -lr * g / (np.abs(g) + eps) + step2, rtol=1e-10)
