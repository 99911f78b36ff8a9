"""B300-native private ring linear algebra (CrypTen's MPC hot path, arXiv 2109.00984).

All protocol arithmetic runs in the CUDA library libmpcring.so (see
include/mpc_ring.h); this package is its Python binding.  The library is
loaded on first use (so that ``python -m paper_2109_00984_b300.build`` can run
before it exists); every entry point raises if it is missing.  There is no
CPU fallback.
"""
from . import _lib
from .api import *  # noqa: F401,F403
from .api import MPCError, PLAIN, LIMB, AUTO, KS_GATES  # noqa: F401


def load_library():
    """Load libmpcring.so now (raises ImportError if it is missing)."""
    return _lib.load()
