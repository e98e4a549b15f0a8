"""GB300 (sm_103a) semiring product and closure library — Python binding.

The computation lives in lib/libsemiring.so (CUDA kernels behind the C ABI of
include/semiring.h).  This package only marshals arguments: _capi is the
one-to-one binding.
"""

from . import _capi
from ._capi import *  # noqa: F401,F403  (the C ABI names)
from ._capi import SemiringError, version  # noqa: F401

__all__ = [n for n in dir(_capi) if not n.startswith("_")]
