"""Pins of the oracle's obstacle cells (the rhomboid obstacles of the Sec. 6
channel).  An obstacle is solid like the wall rows: where a mask reproduces
the wall rows of a walled channel, the run must equal the walled run
exactly; with real obstacles mass is conserved and the fluid inside stays
at rest."""
import numpy as np

import oracle
from workloads import geometry, mesh


def _walls_as_mask(nx, ny, nz):
    m = np.zeros((nz, ny, nx), dtype=bool)
    m[:, 0, :] = True
    m[:, ny - 1, :] = True
    return m


def test_mask_rows_equal_the_walls_exactly():
    nx, ny, nz = 6, 12, 5
    a = oracle.Oracle(nx, ny, nz, walls=True, tau=0.9, body_force=(1e-5, 0, 2e-6))
    b = oracle.Oracle(nx, ny, nz, walls=False, tau=0.9, body_force=(1e-5, 0, 2e-6))
    b.set_solid(_walls_as_mask(nx, ny, nz))
    a.fluid_init()
    b.fluid_init()
    a.step(300)
    b.step(300)
    fa = a.populations()[:, 1:ny - 1]
    fb = b.populations()[:, 1:ny - 1]
    assert np.array_equal(fa, fb)
    assert np.array_equal(a.velocity()[:, :, 1:ny - 1], b.velocity()[:, :, 1:ny - 1])


def test_mask_rows_equal_the_walls_with_an_object_near_them():
    nx, ny, nz = 16, 12, 16
    n1, t1 = mesh.icosphere(1)
    runs = []
    for walls in (True, False):
        o = oracle.Oracle(nx, ny, nz, walls=walls, tau=1.0, body_force=(1e-5, 0, 0), friction=0.05)
        if not walls:
            o.set_solid(_walls_as_mask(nx, ny, nz))
        o.template_create(n1, t1, (2.0, 2.0, 2.0), ks=0.1, kb=0.03, kal=0.1, kag=0.4, kv=1.0)
        o.object_add(0, (8.0, 3.2, 8.0))   # lowest nodes within one cell of the plane y = 1
        o.fluid_init()
        o.step(100)
        runs.append(o)
    xa, xb = runs[0].read_nodes(0)[0], runs[1].read_nodes(0)[0]
    assert np.array_equal(xa, xb)
    assert np.array_equal(runs[0].dropped(), runs[1].dropped()) and np.abs(runs[0].dropped()).max() > 0


def test_obstacles_conserve_mass_and_hold_no_flow():
    nx, ny, nz = 40, 16, 24
    mask = geometry.staggered_rhomboids(nx, ny, nz, count=3, seed=5)
    assert mask.sum() > 100
    o = oracle.Oracle(nx, ny, nz, walls=True, tau=1.0, body_force=(2e-5, 0, 0))
    o.set_solid(mask)
    o.fluid_init()
    m0 = o.fluid_totals()[0]
    o.step(400)
    assert abs(o.fluid_totals()[0] - m0) < 1e-11 * m0
    u = o.velocity()
    assert np.abs(u[:, mask]).max() == 0.0
    # the posts slow the flow: the cells next to them are slower than the
    # same cells of the open channel
    p = oracle.Oracle(nx, ny, nz, walls=True, tau=1.0, body_force=(2e-5, 0, 0))
    p.fluid_init()
    p.step(400)
    assert u[0][~mask].mean() < p.velocity()[0][~mask].mean()
