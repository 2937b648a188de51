"""Learned correction of the ILU(0) factor (binding of the mpk_gnn_* calls of include/mpk.h).

Argument marshalling and the training loop's control flow only: the network's forward and
backward passes, the loss and its gradient, the optimiser step and the correction of the factor
all run in libmpk's CUDA kernels (csrc/gnn.cu).  The network and loss are documented there.
Plain ILU(0) is the fallback (an untrained network returns the plain factor) and the arbiter: see
`solve_with_fallback`.
"""
import ctypes

import numpy as np
import torch

from . import _lib, inputs

NPARAMS = 12193


class Workspace:
    def __init__(self, n, nnz, nprobe=4, nsys=1, device="cuda"):
        nbytes = int(_lib.lib().mpk_gnn_workspace_bytes(n, nnz, nprobe, nsys))
        if nbytes == 0:
            raise ValueError("bad workspace request")
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.nbytes = nbytes


class LearnedILU:
    """Network parameters and Adam state on the device."""

    def __init__(self, params=None, seed=2504_14498 + 5, device="cuda"):
        L = _lib.lib()
        assert L.mpk_gnn_nparams() == NPARAMS
        P = inputs.gnn_init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        self.params = torch.as_tensor(P, device=device).clone()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0

    def forward(self, A, M, ws, o=None):
        o = torch.empty(A.nnz, dtype=torch.float32, device=self.params.device) if o is None else o
        _lib._check(_lib.lib().mpk_gnn_forward(ctypes.byref(A.desc), M.handle, _lib._ptr(self.params), _lib._ptr(o),
                                               _lib._ptr(ws.buf), ws.nbytes, _lib._stream()))
        return o

    def loss(self, A, M, o, probes, ws, sys_rows=None, kind="precond"):
        """(loss, g_o) of the corrected factor; probes: n x nprobe binary32 device tensor.
        kind 'precond': ||M'^-1 A W - W||^2 / ||W||^2 (the training loss); 'factor':
        ||(L'U' - A) W||^2 / ||A W||^2."""
        nprobe = probes.shape[1]
        loss = torch.empty(1, dtype=torch.float32, device=o.device)
        go = torch.empty_like(o)
        nsys, rows = 1, None
        if sys_rows is not None:
            rows = torch.as_tensor(np.asarray(sys_rows, dtype=np.int32), device=o.device)
            nsys = rows.numel() - 1
        fn = _lib.lib().mpk_gnn_loss_precond if kind == "precond" else _lib.lib().mpk_gnn_loss
        _lib._check(fn(ctypes.byref(A.desc), M.handle, _lib._ptr(o), nprobe,
                                            _lib._ptr(probes), nsys, _lib._ptr(rows) if rows is not None else None,
                                            _lib._ptr(loss), _lib._ptr(go), _lib._ptr(ws.buf), ws.nbytes,
                                            _lib._stream()))
        return loss, go

    def backward(self, A, M, go, ws):
        _lib._check(_lib.lib().mpk_gnn_backward(ctypes.byref(A.desc), M.handle, _lib._ptr(self.params), _lib._ptr(go),
                                                _lib._ptr(self.grad), _lib._ptr(ws.buf), ws.nbytes, _lib._stream()))
        return self.grad

    def adam(self, lr):
        self.step += 1
        _lib._check(_lib.lib().mpk_gnn_adam(NPARAMS, _lib._ptr(self.params), _lib._ptr(self.grad), _lib._ptr(self.m),
                                            _lib._ptr(self.v), float(lr), self.step, _lib._stream()))

    def train_step(self, A, M, probes, ws, sys_rows=None, lr=1e-3, kind="precond"):
        o = self.forward(A, M, ws)
        loss, go = self.loss(A, M, o, probes, ws, sys_rows, kind)
        self.backward(A, M, go, ws)
        self.adam(lr)
        return loss

    def correct(self, A, M, ws=None):
        """Replace M's factor by the corrected factor (in M's precision)."""
        ws = ws or Workspace(A.n, A.nnz, 1, 1, device=self.params.device)
        o = self.forward(A, M, ws)
        _lib._check(_lib.lib().mpk_ilu0_correct(M.handle, _lib._ptr(o), _lib._stream()))
        return M


def solve_with_fallback(method, w, A, M_plain, M_learned, b, **kw):
    """Solve with the learned factor and with the plain one; plain ILU(0) judges: the learned
    result is kept only if it converged in no more iterations and reached the same true-residual
    level.  Returns (chosen, learned, plain)."""
    lr = _lib.krylov_solve(method, w, A, M_learned, b, **kw)
    pl = _lib.krylov_solve(method, w, A, M_plain, b, **kw)
    ok = lr["status"] == "OK" and lr["iters"] <= pl["iters"] and lr["relres_true"] <= max(pl["relres_true"] * 10, 1e-300)
    return (lr if ok else pl), lr, pl
