"""Seeded obstacle geometry for channel scenes (input data only).

``rhomboid_mask`` rasterises ESPResSo-style rhomboids (the obstacles of the
paper's Sec. 6 channel, built there with ``constraint rhomboid`` /
``lbboundary rhomboid``): the parallelepiped corner + s a + t b + u c,
s, t, u in [0, 1].  A lattice cell (i, j, k), whose node sits at
(i + 1/2, j + 1/2, k + 1/2), is solid when its node lies inside.  The
paper's geometry file is not available; ``staggered_rhomboids`` places a
seeded row of slanted obstacles in a channel as a stand-in.
"""
from __future__ import annotations

import numpy as np


def rhomboid_mask(shape_zyx, corner, a, b, c, mask=None):
    nz, ny, nx = shape_zyx
    if mask is None:
        mask = np.zeros(shape_zyx, dtype=bool)
    M = np.array([a, b, c], dtype=np.float64).T  # columns a, b, c
    Minv = np.linalg.inv(M)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    p = np.stack([x, y, z], axis=-1) - np.asarray(corner, dtype=np.float64)
    st = p @ Minv.T
    inside = np.all((st >= 0.0) & (st <= 1.0), axis=-1)
    mask |= inside
    return mask


def staggered_rhomboids(nx, ny, nz, count=3, seed=5, height=None):
    """`count` slanted rhomboid posts across the channel (walls at y = 0 and
    ny - 1), evenly spaced along x with seeded offsets; each spans the
    fluid rows."""
    rng = np.random.default_rng(seed)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    h = float(ny - 2) if height is None else float(height)
    for i in range(count):
        x0 = (i + 0.5) * nx / count - 2.0 + rng.uniform(-1.0, 1.0)
        z0 = rng.uniform(0.2, 0.6) * nz
        rhomboid_mask((nz, ny, nx), (x0, 1.0, z0), (3.0, 0.0, 0.0), (0.0, h, 0.0),
                      (rng.uniform(-2.0, 2.0), 0.0, rng.uniform(3.0, 0.25 * nz)), mask)
    return mask
