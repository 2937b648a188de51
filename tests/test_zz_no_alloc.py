"""mpk_dot_noalloc: the inner product for callers that must not let the library allocate device
memory (fixed scratch inside the library).  Collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test.

It must reproduce mpk_dot exactly (same kernel, same fixed summation order), also on a second
call that finds the previous call's leftovers in the shared scratch, and reject lengths above
its fixed limit.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2504_14498_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

MAX_N = 16777216  # MPK_DOT_NOALLOC_MAX_N in include/mpk.h


def _call(fn, n, c, w, a, b, out):
    L = _lib.lib()
    st = getattr(L, fn)(n, int(c == 2), w, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("w,c,n", [(2, 1, 1000003), (1, 1, 4097), (4, 2, 70001), (3, 1, 33)])
def test_noalloc_matches_dot_twice(w, c, n):
    a = torch.as_tensor(inputs.random_vector(n, w, c, seed=61), device="cuda")
    b = torch.as_tensor(inputs.random_vector(n, w, c, seed=62), device="cuda")
    ref = torch.empty(c * w, dtype=torch.float64, device="cuda")
    assert _call("mpk_dot", n, c, w, a, b, ref) == 0
    for _ in range(2):  # the second call sees the first call's leftovers in the shared scratch
        out = torch.full((c * w,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call("mpk_dot_noalloc", n, c, w, a, b, out) == 0
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_oversize():
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _call("mpk_dot_noalloc", MAX_N + 1, 1, 2, a, a, out) == 6  # MPK_INVALID_ARG, nothing launched
    assert b"exceeds" in _lib.lib().mpk_last_error()
