"""Learned ILU(0) correction on the GPU against the oracle (oracle/gnn.py).

Bars (binary32 arithmetic and bfloat16-stored activations on the GPU, binary64 with emulated
bfloat16 rounding in the oracle; the summation orders differ):
  * network output o: within 2e-2 of max |o| per entry;
  * loss: within 1e-4 relative; d loss / d o: within 1e-3 relative (2-norm);
  * d loss / d parameters: within 3e-2 relative (2-norm), cosine >= 0.999;
  * one Adam step: within 1e-5 relative;
  * the corrected factor: the library's tanh in binary32, within 1e-6 relative; the repacked
    factor then substitutes bit for bit like the oracle given the same values.
A short training run shows what the network gains over plain ILU(0), which judges it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import gnn
from paper_2504_14498_gb300 import _lib, inputs, learned

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _params(seed=1):
    P = inputs.gnn_init_params(seed)
    rng = np.random.default_rng(seed + 100)
    P[gnn.P_DEC + gnn.D_WO:gnn.P_DEC + gnn.D_BO] = rng.uniform(-0.3, 0.3, gnn.H).astype(np.float32)
    P[gnn.P_DEC + gnn.D_BO] = 0.05
    return P


def _setup(m=24, seed=3, prec="fp32"):
    A_t = inputs.convdiff2d_random(m, seed)
    A = _lib.Matrix.from_tuple(A_t)
    M = _lib.ILU0(A, prec)
    st, fac, _ = oracle.ilu0(A_t, prec)
    assert st == 0
    return A_t, A, M, fac


def test_forward_loss_backward_match_oracle():
    A_t, A, M, fac = _setup()
    P = _params()
    net = learned.LearnedILU(P)
    K = 4
    W = inputs.probe_vectors(A_t[0], K, 8)
    ws = learned.Workspace(A.n, A.nnz, K, 1)
    o = net.forward(A, M, ws)
    o_ref, cache = gnn.forward(P.astype(np.float64), A_t, fac)
    og = host(o).astype(np.float64)
    assert np.max(np.abs(og - o_ref)) <= 2e-2 * np.max(np.abs(o_ref)) + 1e-4
    loss, go = net.loss(A, M, o, dev(W, torch.float32), ws, kind="factor")
    L_ref, go_ref = gnn.loss(A_t, fac, og, W)  # the oracle's loss of the GPU's own o
    assert abs(float(host(loss)[0]) - L_ref) <= 1e-4 * L_ref
    gog = host(go).astype(np.float64)
    assert np.linalg.norm(gog - go_ref) <= 1e-3 * np.linalg.norm(go_ref)
    G = host(net.backward(A, M, go, ws)).astype(np.float64)
    G_ref = gnn.backward(P.astype(np.float64), A_t, cache, gog)
    assert np.linalg.norm(G - G_ref) <= 3e-2 * np.linalg.norm(G_ref)
    assert G @ G_ref >= 0.999 * np.linalg.norm(G) * np.linalg.norm(G_ref)


def test_batched_loss_matches_oracle():
    sys_ = [inputs.convdiff2d_random(m, 40 + m) for m in (10, 13, 16)]
    B_t, roff = inputs.block_diagonal(sys_)
    B_t = (B_t[0], B_t[1].astype(np.int32), B_t[2], B_t[3])
    B = _lib.Matrix.from_tuple(B_t)
    M = _lib.ILU0(B, "fp32")
    _, fac, _ = oracle.ilu0(B_t, "fp32")
    K = 3
    W = inputs.probe_vectors(B_t[0], K, 2)
    o = np.random.default_rng(5).uniform(-1, 1, len(B_t[2])).astype(np.float32)
    net = learned.LearnedILU(_params())
    ws = learned.Workspace(B.n, B.nnz, K, len(sys_))
    for kind, ref_fn in (("factor", gnn.loss), ("precond", gnn.loss_precond)):
        loss, go = net.loss(B, M, dev(o, torch.float32), dev(W, torch.float32), ws, roff, kind=kind)
        L_ref, go_ref = ref_fn(B_t, fac, o.astype(np.float64), W, roff)
        assert abs(float(host(loss)[0]) - L_ref) <= 1e-4 * L_ref, kind
        assert np.linalg.norm(host(go) - go_ref) <= 2e-3 * np.linalg.norm(go_ref), kind


def test_precond_loss_matches_oracle_and_rejects_unsymmetric():
    A_t, A, M, fac = _setup(m=30, seed=12)
    K = 4
    W = inputs.probe_vectors(A_t[0], K, 3)
    o = np.random.default_rng(9).uniform(-1, 1, len(A_t[2])).astype(np.float32)
    net = learned.LearnedILU(_params())
    ws = learned.Workspace(A.n, A.nnz, K, 1)
    loss, go = net.loss(A, M, dev(o, torch.float32), dev(W, torch.float32), ws)
    L_ref, go_ref = gnn.loss_precond(A_t, fac, o.astype(np.float64), W)
    assert abs(float(host(loss)[0]) - L_ref) <= 1e-4 * L_ref
    assert np.linalg.norm(host(go) - go_ref) <= 2e-3 * np.linalg.norm(go_ref)
    R_t = inputs.random_sparse(200, 3, 9, seed=4)  # unsymmetric pattern: refused before any solve
    R = _lib.Matrix.from_tuple(R_t)
    wr = learned.Workspace(R.n, R.nnz, 2, 1)
    with pytest.raises(_lib.MpkError) as e:
        net.loss(R, _lib.ILU0(R, "fp32"), torch.zeros(R.nnz, device="cuda"),
                 dev(inputs.probe_vectors(200, 2, 1), torch.float32), wr)
    assert e.value.status == "INVALID_ARG"


def test_adam_step_matches_formula():
    rng = np.random.default_rng(2)
    net = learned.LearnedILU(rng.standard_normal(learned.NPARAMS).astype(np.float32))
    P0 = host(net.params).astype(np.float64)
    m, v = np.zeros_like(P0), np.zeros_like(P0)
    for step in range(1, 4):
        g = rng.standard_normal(learned.NPARAMS).astype(np.float32)
        net.grad.copy_(dev(g, torch.float32))
        net.adam(1e-2)
        P0, m, v = gnn.adam(P0, g.astype(np.float64), m, v, 1e-2, step)
        assert np.max(np.abs(host(net.params) - P0)) <= 1e-5 * np.max(np.abs(P0))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_correction_and_repacked_substitution(prec):
    A_t, A, M, fac = _setup(m=20, seed=7, prec=prec)
    net = learned.LearnedILU(_params(4))
    net.correct(A, M)
    got = host(M.values())
    ws = learned.Workspace(A.n, A.nnz, 1, 1)
    o = host(net.forward(A, _lib.ILU0(A, prec), ws)).astype(np.float64)
    ref = gnn.corrected(fac, o)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)) <= (1e-6 if prec == "fp64" else 5e-7)
    r = inputs.random_vector(A_t[0], 2, 1, seed=9)
    for trans in (False, True):
        z = host(M.apply(dev(r), 2, trans))
        assert np.array_equal(z, oracle.precond(A_t, got, r, 2, prec, 1, trans))


def _batch_of(ms, seeds):
    sys_ = [inputs.convdiff2d_random(m, s) for m, s in zip(ms, seeds)]
    B_t, roff = inputs.block_diagonal(sys_)
    return sys_, (B_t[0], B_t[1].astype(np.int32), B_t[2], B_t[3]), roff


def test_training_reduces_loss_and_iterations_are_judged():
    """Train on 48 seeded 32x32 instances (6 batches of 8, 25 epochs, loss of the preconditioned
    operator over half smooth, half random probes) and evaluate on 6 held-out 48x48 instances with
    DD BiCGSTAB + binary64 ILU(0): the loss must fall, and the arbitrated result (learned factor kept
    only when it needs no more iterations) never needs more than plain.  The training at the
    workload's scale is bench.py --workload learned."""
    net = learned.LearnedILU(seed=11)
    K = 4
    batches = []
    for b in range(6):
        _, B_t, roff = _batch_of([32] * 8, [1000 + 8 * b + k for k in range(8)])
        B = _lib.Matrix.from_tuple(B_t)
        batches.append((B, _lib.ILU0(B, "fp32"), roff, dev(inputs.training_probes(32, 8, K, 77 + b), torch.float32),
                        learned.Workspace(B.n, B.nnz, K, 8)))
    losses = []
    for epoch in range(25):
        for B, M, roff, W, ws in batches:
            losses.append(float(host(net.train_step(B, M, W, ws, roff, lr=3e-3))[0]))
    first, last = np.mean(losses[:6]), np.mean(losses[-6:])
    assert last < 0.97 * first, (first, last)
    gains = []
    for s in range(6):
        A_t = inputs.convdiff2d_random(48, 5000 + s)
        A = _lib.Matrix.from_tuple(A_t)
        b = _lib.spmv_mp(A, dev(inputs.ones(A_t[0], 2)), 2)
        Mp = _lib.ILU0(A, "fp64")
        Ml = net.correct(A, _lib.ILU0(A, "fp64"))
        chosen, lr_, pl = learned.solve_with_fallback("bicgstab", 2, A, Mp, Ml, b, tol_rel=1e-25, maxit=600)
        assert pl["status"] == "OK" and chosen["status"] == "OK"
        assert chosen["iters"] <= pl["iters"]
        gains.append(pl["iters"] - lr_["iters"])
    print("training loss %.4f -> %.4f; held-out iteration gains (plain - learned): %s" % (first, last, gains))
