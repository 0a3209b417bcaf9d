"""GB300-native Krylov cone-beam CT reconstruction (after arXiv 2211.14212).

libcbct.so (built from csrc/ by ``build.build()``) holds the Siddon forward
projector, its exact transpose and the CGLS / LSQR / LSMR / hybrid-LSQR
solvers as sm_103a CUDA kernels behind the C ABI of include/cbct.h;
``cbct`` is its Python binding.
"""
from . import cbct  # noqa: F401

__all__ = ["cbct"]
