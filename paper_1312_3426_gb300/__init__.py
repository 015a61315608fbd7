"""GB300-native lattice-Boltzmann / immersed-boundary step (arXiv:1312.3426).

The computation runs in the CUDA library ``_lbib.so`` built from ``csrc/``
(see ``build.py``); ``lbib`` is its thin ctypes binding.  Importing this
package does not build anything; ``lbib.load()`` raises when the library is
missing.
"""
from . import lbib  # noqa: F401
from .lbib import LbibError, Sim  # noqa: F401

__all__ = ["lbib", "Sim", "LbibError"]
