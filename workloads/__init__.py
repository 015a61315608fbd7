"""Seeded synthetic inputs shared by the oracle and the CUDA library.

Holds meshes and scene recipes only; no part of the method's arithmetic.
"""
from . import mesh, scenes  # noqa: F401
