"""GB300 (sm_103a) state-vector gate engine after arXiv 2001.10554 (Intel Quantum Simulator).

The computation lives in the CUDA library ``libiqsgpu.so`` (C ABI in
``include/iqs.h``); this package only marshals arguments to it.  Importing
it fails if the library has not been built -- there is no CPU fallback.
"""
from ._lib import IQS_C64, IQS_C128, IQSError, version  # noqa: F401
from .register import Register, mat8  # noqa: F401
from .qaoa import QAOA  # noqa: F401
from .pool import Pool, PoolMany  # noqa: F401

__all__ = ["Register", "QAOA", "Pool", "PoolMany", "IQSError", "IQS_C64", "IQS_C128", "version", "mat8"]
