"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/mpk.h
declares (no GPU needed: nothing is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpk.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libmpk():
    from paper_2504_14498_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("mpk_spmv_mp", "mpk_ilu0_factor", "mpk_krylov_solve", "mpk_precond_apply", "mpk_dot"):
        assert required in names


def test_every_declared_symbol_is_exported(libmpk):
    missing = [n for n in _declared() if not hasattr(libmpk, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2504_14498_gb300 import _lib

    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert set(_declared()) <= bound, set(_declared()) - bound


def test_version_and_error_without_gpu(libmpk):
    libmpk.mpk_version.restype = ctypes.c_int
    assert libmpk.mpk_version() >= 100
    libmpk.mpk_last_error.restype = ctypes.c_char_p
    assert isinstance(libmpk.mpk_last_error(), bytes)


def test_invalid_arguments_rejected_on_host(libmpk):
    """Argument checks happen before any CUDA call, so they work without a GPU."""
    from paper_2504_14498_gb300 import _lib

    L = _lib.lib()
    assert L.mpk_spmv_mp(None, 2, None, None, None) == 6
    assert L.mpk_dot(0, 0, 2, None, None, None, None) == 6
    assert L.mpk_ilu0_factor(None, 0, None, None, None) == 6
    d = _lib.CsrDesc(0, 0, None, None, None, 0)
    h = ctypes.c_void_p()
    assert L.mpk_ilu0_factor(ctypes.byref(d), 0, ctypes.byref(h), None, None) == 6
    assert L.mpk_krylov_solve(7, 2, ctypes.byref(d), None, None, None, None, None, None) == 6
    assert L.mpk_ilu0_levels(None, 0, None, None, None) == 6


def test_oracle_and_library_share_no_code():
    """The CUDA sources never include or reference the oracle, and vice versa."""
    csrc = os.path.join(ROOT, "paper_2504_14498_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    otxt = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "mp.cuh" not in otxt and "mpk.h" not in otxt


def test_binding_refuses_host_and_malformed_tensors():
    """The binding passes raw device pointers: a host tensor, a strided view, a non-tensor or a
    short or narrower buffer is refused with ValueError before any call reaches the library."""
    import torch

    from paper_2504_14498_gb300 import _lib

    with pytest.raises(ValueError, match="device memory"):
        _lib._ptr(torch.zeros(4))
    with pytest.raises(ValueError, match="torch tensor"):
        _lib._ptr([0.0, 1.0])

    class FakeA:  # only what spmv_mp reads before marshalling
        n, cp, desc = 3, 1, None

    with pytest.raises(ValueError, match="device memory"):
        _lib.spmv_mp(FakeA(), torch.zeros(6, dtype=torch.float64), 2)
    with pytest.raises(ValueError, match="device memory"):
        _lib.dot(torch.zeros(6, dtype=torch.float64), torch.zeros(6, dtype=torch.float64), 3, 2)


def test_misaligned_device_pointers_refused_before_any_launch(libmpk):
    """Vectors (and complex matrix values) are accessed 16 bytes at a time, so every entry point
    refuses a misaligned device pointer with MPK_INVALID_ARG (6) before it queues any work: the
    fake addresses below are never dereferenced, here or on a GPU."""
    from paper_2504_14498_gb300._lib import CsrDesc, Info, Opts

    vp = ctypes.c_void_p
    bad, good = vp(0x100008), vp(0x200000)
    libmpk.mpk_last_error.restype = ctypes.c_char_p
    A = CsrDesc(4, 0, good, good, good, 0)
    Ac = CsrDesc(4, 0, good, good, bad, 1)  # complex values misaligned
    opts = Opts(1e-10, 0.0, 10, 1, 0, 0, None, None)
    info = Info()
    calls = [
        ("mpk_spmv_mp", lambda: libmpk.mpk_spmv_mp(ctypes.byref(A), 2, bad, good, None)),
        ("mpk_spmv_mp y", lambda: libmpk.mpk_spmv_mp(ctypes.byref(A), 2, good, bad, None)),
        ("mpk_spmv_mp complex val", lambda: libmpk.mpk_spmv_mp(ctypes.byref(Ac), 2, good, vp(0x300000), None)),
        ("mpk_dot", lambda: libmpk.mpk_dot(8, 0, 2, good, bad, vp(0x300000), None)),
        ("mpk_dot_noalloc", lambda: libmpk.mpk_dot_noalloc(8, 0, 2, bad, good, vp(0x300000), None)),
        ("mpk_mp_op", lambda: libmpk.mpk_mp_op(0, 2, 4, good, good, bad, None)),
        ("mpk_krylov_solve", lambda: libmpk.mpk_krylov_solve(2, 2, ctypes.byref(A), None, bad, good,
                                                             ctypes.byref(opts), ctypes.byref(info), None)),
        ("mpk_krylov_solve complex val", lambda: libmpk.mpk_krylov_solve(2, 2, ctypes.byref(Ac), None, good,
                                                                         vp(0x300000), ctypes.byref(opts),
                                                                         ctypes.byref(info), None)),
        ("mpk_ilu0_factor complex val", lambda: libmpk.mpk_ilu0_factor(ctypes.byref(Ac), 1, ctypes.byref(vp()),
                                                                       None, None)),
    ]
    for name, call in calls:
        assert call() == 6, name
        assert b"16-byte aligned" in libmpk.mpk_last_error(), name
