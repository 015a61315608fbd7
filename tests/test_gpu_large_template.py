"""The largest template class: one sphere of 4098 nodes (the octahedron
subdivided five times, 8192 triangles, radius 11 lu; 181 KB of shared memory
for its staged positions and forces, near the 227 KB a block can hold),
deformed at the start so that all five membrane forces act, in a walled
channel with a body force, 300 steps against the FP64 oracle.  Launch
shapes: one block per object; a cluster of two blocks per object; and a
request for four objects per block, which the library lowers to the one
that fits.  Bars as stated for the method: velocity 1e-5 relative L2, nodes
1e-6 lu.
"""
import numpy as np
import pytest

import oracle
from paper_1312_3426_gb300 import lbib
from workloads import mesh, scenes

pytestmark = pytest.mark.gpu

STEPS = 300


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_3426_gb300 import build
    build.build()
    lbib.load()


def scene():
    sc = scenes.Scene("sphere4098_40x32x40", 40, 32, 40, steps=STEPS)
    nodes, tris = mesh.octasphere(5)
    sc.templates.append(scenes.Template(nodes, tris, (11.0, 11.0, 11.0), **scenes.PAPER_MODULI))
    sc.objects.append(scenes.Obj(0, (20.0, 16.0, 20.0)))
    return sc


@pytest.fixture(scope="module")
def reference():
    sc = scene()
    o = oracle.Oracle.from_scene(sc)
    X, _ = o.read_nodes(0)
    c = X.mean(0)
    Xd = c + (X - c) * np.array([1.05, 1.0 / 1.05, 1.0])
    o.object_set_nodes(0, Xd)
    o.step(STEPS)
    return sc, Xd, o.velocity(), o.read_nodes(0)[0]


@pytest.mark.parametrize("cluster,group", [(1, 1), (2, 1), (1, 4)])
def test_largest_template_matches_oracle(reference, cluster, group):
    sc, Xd, uo, xo = reference
    g = lbib.Sim.from_scene(sc)
    lbib.lbib_set_tuning(g.h, lbib.LBIB_TUNE_IB_CLUSTER, cluster)
    lbib.lbib_set_tuning(g.h, lbib.LBIB_TUNE_MEMBRANE_GROUP, group)
    g.object_set_nodes(0, Xd)
    g.step(STEPS)
    g.sync()
    ug = g.velocity()
    xg = g.read_nodes(0)[0]
    g.close()
    rows = slice(1, sc.ny - 1)
    err_u = float(np.linalg.norm(ug[:, :, rows, :].astype(np.float64) - uo[:, :, rows, :]) /
                  np.linalg.norm(uo[:, :, rows, :]))
    err_x = float(np.abs(xg - xo).max())
    moved = float(np.abs(xo - Xd).max())
    print(f"\n4098-node sphere, {STEPS} steps, cluster {cluster}, group {group}: velocity rel L2 {err_u:.3e}, "
          f"node max-abs {err_x:.3e} lu (nodes moved up to {moved:.3e} lu)")
    assert moved > 0.05
    assert err_u <= 1e-5, err_u
    assert err_x <= 1e-6, err_x
