"""Slab decomposition of one channel along x over R ranks (Sec. 2 fluid,
one lattice step per exchange).

Every run of this package holds one simulation per GPU and scales by
independent replicas, so no kernel uses this; it fixes the indexing that a
decomposed run would use, and is exercised by CPU ranks (gloo) against the
undecomposed step.

Rank r owns the x planes [x0, x1) (balanced, contiguous, periodic order of
ranks) and keeps one ghost plane on each side: local plane 0 is global
x0 - 1, local planes 1..n are x0..x1-1, local plane n+1 is x1 (periodic).
A pull-scheme step needs, across each face, only the populations that move
across it: the 5 directions with e_x = +1 from the left neighbour's last
plane and the 5 with e_x = -1 from the right neighbour's first plane
(`crossing_directions`).  A push-scheme step (post-collision values pushed
to the neighbours) collides the ghost planes too, so there the whole plane
state is exchanged (`ghost_sources`).
"""
from __future__ import annotations

import numpy as np


def slab_bounds(nx: int, rank: int, world: int) -> tuple[int, int]:
    """Planes [x0, x1) of `rank`: the first nx % world ranks take one extra."""
    if world < 1 or not 0 <= rank < world or nx < world:
        raise ValueError("need 0 <= rank < world <= nx")
    base, extra = divmod(nx, world)
    x0 = rank * base + min(rank, extra)
    return x0, x0 + base + (1 if rank < extra else 0)


def neighbours(rank: int, world: int) -> tuple[int, int]:
    """(left, right) ranks in the periodic x order."""
    return (rank - 1) % world, (rank + 1) % world


def ghost_sources(nx: int, rank: int, world: int) -> tuple[int, int]:
    """Global x planes the two ghost planes of `rank` mirror: (x0 - 1, x1), periodic."""
    x0, x1 = slab_bounds(nx, rank, world)
    return (x0 - 1) % nx, x1 % nx


def crossing_directions(e: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Directions that cross a face of the slab in a pull step: from the left
    neighbour (e_x = +1) and from the right neighbour (e_x = -1)."""
    e = np.asarray(e)
    return np.flatnonzero(e[:, 0] == 1), np.flatnonzero(e[:, 0] == -1)


def ghosted(full: np.ndarray, nx: int, rank: int, world: int, axis: int) -> np.ndarray:
    """The slab of `rank` with its two ghost planes, cut from an array whose
    `axis` is x (length nx)."""
    x0, x1 = slab_bounds(nx, rank, world)
    idx = np.arange(x0 - 1, x1 + 1) % nx
    return np.take(full, idx, axis=axis)
