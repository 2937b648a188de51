"""GB300 (sm_103a) mixed-precision ILU(0)-preconditioned multi-component Krylov solvers.

Implements the hot path of Kouya, "Assessing the Performance of Mixed-Precision
ILU(0)-Preconditioned Multiple-Precision Real and Complex Krylov Subspace Methods"
(arXiv 2504.14498): D/DD/TD/QD vectors, binary64 CSR matrices, ILU(0) in binary64 / binary32 /
bfloat16, BiCG, CGS, BiCGSTAB and GPBiCG, real and complex.

The compute runs in libmpk.so (C ABI in include/mpk.h, CUDA kernels in csrc/); this package
holds the ctypes binding (_lib), the in-tree build (build) and the synthetic input generators
(inputs).  Submodules are imported lazily so that `inputs` is usable without CUDA.
"""
import importlib

__all__ = ["Matrix", "ILU0", "spmv_mp", "dot", "krylov_solve", "krylov_solve_batched", "solve_host", "MpkError",
           "build", "inputs"]


def __getattr__(name):
    if name in ("build", "inputs"):
        return importlib.import_module("." + name, __name__)
    if name in __all__:
        return getattr(importlib.import_module("._lib", __name__), name)
    raise AttributeError(name)
