"""GB300 (sm_103a) chemical-potential multiphase lattice Boltzmann library.

The compute path is liblbm.so (hand-written CUDA behind the C ABI of
include/lbm.h); this package is its thin Python binding.
"""
from .build import build  # noqa: F401


def load():
    """Return the ctypes binding module (raises ImportError if liblbm.so is missing)."""
    from . import lbm
    lbm.lib()
    return lbm
