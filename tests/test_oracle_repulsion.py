"""Pins of the oracle's soft-sphere repulsion (Sec. 6 interactions; the
potential V(r) = a r^-n below the cutoff is the reading stated in the
oracle).  Closed forms on single node pairs, Newton's third law, the
cutoff, the minimum image across periodic faces and the wall term."""
import numpy as np
import pytest

import oracle
from workloads import mesh

# a small closed mesh (octahedron, inward triangles) used as a rigid probe
NODES, TRIS = mesh.icosphere(0)


def _two(nx=20, ny=12, nz=20, walls=True, sep=(3.0, 0, 0), scale=0.5, base=(6.0, 6.0, 6.0)):
    o = oracle.Oracle(nx, ny, nz, walls=walls, tau=1.0)
    o.template_create(NODES, TRIS, (scale, scale, scale))
    o.object_add(0, base)
    o.object_add(0, tuple(b + s for b, s in zip(base, sep)))
    return o


def _pairs(X, Y, box=None):
    out = []
    for i, a in enumerate(X):
        for j, b in enumerate(Y):
            d = a - b
            if box is not None:
                d = d - box * np.round(d / box)
            out.append((i, j, d))
    return out


def test_single_pair_closed_form_and_third_law():
    a, n, rc = 0.005, 2.0, 0.3
    # two icosahedra of radius 0.5 (x extent +-0.425) whose nearest
    # vertices are 0.2 apart
    o = _two(sep=(1.05, 0.0, 0.0))
    o.set_repulsion((a, n, rc), (0.0, 1.0, 0.0))
    XA, _ = o.read_nodes(0)
    XB, _ = o.read_nodes(1)
    F = o.repulsion_forces()
    exp = np.zeros_like(F)
    nA = len(XA)
    hits = 0
    for i, j, d in _pairs(XA, XB):
        r = np.linalg.norm(d)
        if r < rc:
            hits += 1
            f = a * n * r ** -(n + 1) * d / r
            exp[i] += f
            exp[nA + j] -= f
    assert hits >= 1
    assert np.allclose(F, exp, rtol=1e-14, atol=0)
    assert np.abs(F.sum(0)).max() < 1e-15 * np.abs(F).max()


def test_nothing_beyond_cutoff_and_nothing_within_an_object():
    o = _two(sep=(3.0, 0.0, 0.0))
    o.set_repulsion((0.005, 2.0, 0.3), (0.0, 1.0, 0.0))
    assert np.count_nonzero(o.repulsion_forces()) == 0  # nodes of one object are 0.5 apart: not repelled


def test_minimum_image_across_the_periodic_face():
    # object 0 at x = 0.3, object 1 at x = 19.25 (image -0.75): nearest
    # vertices 0.2 apart through the face x = 0
    o = _two(nx=20, sep=(18.95, 0.0, 0.0), base=(0.3, 6.0, 6.0))
    o.set_repulsion((0.005, 2.0, 0.3), (0.0, 1.0, 0.0))
    F = o.repulsion_forces()
    XA, _ = o.read_nodes(0)
    XB, _ = o.read_nodes(1)
    box = np.array([20.0, 1e300, 20.0])
    exp = np.zeros_like(F)
    for i, j, d in _pairs(XA, XB, box):
        r = np.linalg.norm(d)
        if r < 0.3:
            f = 0.005 * 2.0 * r ** -3.0 * d / r
            exp[i] += f
            exp[len(XA) + j] -= f
    assert np.abs(exp).max() > 0
    assert np.allclose(F, exp, rtol=1e-14, atol=0)
    # the pair pushes object 0 towards +x (away from its image neighbour at x < 0)
    assert F[:len(XA), 0].sum() > 0


def test_wall_term_closed_form():
    a, n, rc = 0.0001, 1.2, 0.6
    o = oracle.Oracle(12, 12, 12, walls=True, tau=1.0)
    o.template_create(NODES, TRIS, (0.5, 0.5, 0.5))
    o.object_add(0, (6.0, 1.9, 6.0))   # lowest vertex at y = 1.4 (0.4 above the wall plane y = 1)
    o.set_repulsion((0.0, 1.0, 0.0), (a, n, rc))
    X, _ = o.read_nodes(0)
    F = o.repulsion_forces()
    for i, x in enumerate(X):
        d = x[1] - 1.0
        want = a * n * d ** -(n + 1) if d < rc else 0.0
        assert F[i, 1] == pytest.approx(want, rel=1e-14, abs=0)
        assert F[i, 0] == 0.0 and F[i, 2] == 0.0
    assert F[:, 1].max() > 0


def test_repulsion_keeps_approaching_objects_apart():
    """Two objects driven into each other by external forces, no fluid
    motion (frozen fluid): with repulsion their nearest nodes stay beyond
    a minimum distance, without it they pass through each other."""
    def closest(o):
        XA, _ = o.read_nodes(0)
        XB, _ = o.read_nodes(1)
        return min(np.linalg.norm(d) for _, _, d in _pairs(XA, XB))

    res = {}
    for on in (False, True):
        o = _two(nx=24, ny=14, nz=14, sep=(2.0, 0.0, 0.0), base=(10.0, 7.0, 7.0))
        if on:
            o.set_repulsion((0.005, 2.0, 0.3), (0.0, 1.0, 0.0))
        o.object_set_force(0, (2e-3, 0.0, 0.0))
        o.object_set_force(1, (-2e-3, 0.0, 0.0))
        o.fluid_init()
        mind = 1e9
        for _ in range(60):
            o.step_nodes_only(10)
            mind = min(mind, closest(o))
        res[on] = mind
    assert res[True] > 0.15 and res[False] < 0.1, res
