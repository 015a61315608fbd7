"""Seeded, synthetic triangulated meshes for elastic objects.

This module only produces input geometry (node coordinates and triangle
index triples).  It holds none of the method's arithmetic: no forces, no
rest-state measures, no lattice-Boltzmann.  Both the FP64 oracle and the
CUDA library consume its output.

Conventions (paper, Sec. 5 "Template creation"):
  * node ids are the row order of the node array, starting from 0;
  * each triangle (A, B, C) is ordered so that AB x AC points *inside* the
    object;
  * coordinates are centred so that the approximate centre is the origin.

Meshes provided:
  * ``icosphere(level)``: the regular icosahedron refined ``level`` times by
    4-way midpoint subdivision and projected on the unit sphere.  Counts:
    10*4**level + 2 nodes, 20*4**level triangles (level 2: 162/320,
    level 3: 642/1280, level 4: 2562/5120).
  * ``biconcave(level)``: the icosphere mapped onto the red-blood-cell
    profile of Evans & Fung (1972), z(r) = +-(R/2) sqrt(1-rho^2)
    (c0 + c1 rho^2 + c2 rho^4), rho = r/R, with their published constants
    c0 = 0.2072, c1 = 2.0026, c2 = -1.1228.  Unit radius; scale with the
    template ``stretch`` option.
"""
from __future__ import annotations

import numpy as np

# Evans & Fung (1972) biconcave shape constants (published values).
EVANS_FUNG_C0 = 0.2072
EVANS_FUNG_C1 = 2.0026
EVANS_FUNG_C2 = -1.1228


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def _orient_inward(nodes: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Order each triangle of a star-shaped (about the origin) mesh inward."""
    a, b, c = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    n = np.cross(b - a, c - a)
    outward = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) > 0.0
    out = tris.copy()
    out[outward, 1], out[outward, 2] = tris[outward, 2], tris[outward, 1]
    return out


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: (nodes float64 [N,3], triangles int32 [T,3]), inward."""
    if level < 0:
        raise ValueError("level must be >= 0")
    verts, faces = _icosahedron()
    verts = [tuple(p) for p in verts]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            k = cache.get(key)
            if k is None:
                p = np.add(verts[i], verts[j]) * 0.5
                p = p / np.linalg.norm(p)
                verts.append(tuple(p))
                k = len(verts) - 1
                cache[key] = k
            return k

        new = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        faces = np.array(new, dtype=np.int64)
    nodes = np.array(verts, dtype=np.float64)
    tris = _orient_inward(nodes, np.asarray(faces, dtype=np.int64))
    return nodes, tris.astype(np.int32)


def biconcave(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit-radius Evans-Fung red-blood-cell surface (axis along z), inward.

    Each icosphere node (x, y, z) keeps its (x, y); its height becomes
    sign(z) * 0.5 * sqrt(1 - rho^2) * (c0 + c1 rho^2 + c2 rho^4) with
    rho^2 = x^2 + y^2.  Because |z| = sqrt(1 - rho^2) on the unit sphere this
    is a positive rescaling of z, so triangle orientation is preserved.
    """
    nodes, tris = icosphere(level)
    rho2 = np.clip(nodes[:, 0] ** 2 + nodes[:, 1] ** 2, 0.0, 1.0)
    scale = 0.5 * (EVANS_FUNG_C0 + EVANS_FUNG_C1 * rho2 + EVANS_FUNG_C2 * rho2 * rho2)
    out = nodes.copy()
    out[:, 2] = nodes[:, 2] * scale
    return out, tris


def biconcave_volume(radius: float) -> float:
    """Closed-form volume of the Evans-Fung surface of radius R.

    V = 2 pi R^3 int_0^1 sqrt(1-p^2) (c0 + c1 p^2 + c2 p^4) p dp
      = 2 pi R^3 (c0/3 + 2 c1/15 + 8 c2/105).
    """
    k = EVANS_FUNG_C0 / 3.0 + 2.0 * EVANS_FUNG_C1 / 15.0 + 8.0 * EVANS_FUNG_C2 / 105.0
    return 2.0 * np.pi * radius ** 3 * k


def tetrahedron() -> tuple[np.ndarray, np.ndarray]:
    """Regular tetrahedron centred at the origin, inward-oriented."""
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    f = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int64)
    return v, _orient_inward(v, f).astype(np.int32)


def octahedron() -> tuple[np.ndarray, np.ndarray]:
    """Regular octahedron (unit circumradius), inward-oriented."""
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float64)
    f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int64)
    return v, _orient_inward(v, f).astype(np.int32)


def octasphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit sphere from the octahedron by `level` midpoint subdivisions
    (4 * 4^level + 2 nodes, 8 * 4^level triangles; level 5: 4098 nodes,
    near the largest template the library stages), inward-oriented."""
    if level < 0:
        raise ValueError("level must be >= 0")
    v, f = octahedron()
    verts = [tuple(p) for p in v]
    faces = [tuple(int(i) for i in t) for t in f]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            k = cache.get(key)
            if k is None:
                p = np.add(verts[i], verts[j]) * 0.5
                verts.append(tuple(p / np.linalg.norm(p)))
                k = len(verts) - 1
                cache[key] = k
            return k

        new = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new
    nodes = np.array(verts, dtype=np.float64)
    tris = _orient_inward(nodes, np.asarray(faces, dtype=np.int64))
    return nodes, tris.astype(np.int32)
