"""libsfhad: the sum-factorized Hadamard-product volume term of entropy-
conserving flux differencing (arXiv 2306.11665), GB300-native.

* ``_abi``    -- ctypes binding of include/sfhad.h (same function names)
* ``api``     -- torch helpers: Context, volume_residual, vjp, SFHVolume
* ``inputs``  -- seeded synthetic meshes, metric terms and states
* ``build``   -- nvcc build of libsfhad.so for sm_103a
"""
from . import _abi  # noqa: F401
from ._abi import SfhError  # noqa: F401

__version__ = "1.0.0"
