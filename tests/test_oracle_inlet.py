"""Pins of the oracle's velocity inlet (Sec. 6: the example sets the fluid
velocity of the inflow plane before every step).  Reading: the inlet
replaces the populations of its cells by the equilibrium at the cell's own
density and the prescribed velocity."""
import numpy as np

import oracle

U = np.array([0.0, 0.0, 0.01])


def test_inlet_cells_carry_the_prescribed_velocity_and_keep_their_density():
    o = oracle.Oracle(8, 10, 12, walls=True, tau=0.9)
    o.set_inlet((1, 7, 1, 9, 1, 2), U)   # the plane z = 1 inside the walls, as in the example
    o.fluid_init()
    o.step(30)
    # let the flow develop, then one more step: the collision's velocity at
    # the inlet cells is the prescribed one (no body force), whatever came in
    u = o.velocity()
    assert np.abs(u[:, 1, 1:9, 1:7] - U[:, None, None]).max() < 1e-15
    # outside the inlet the flow has been driven
    assert u[2, 3, 5, 4] > 1e-5
    # the inlet keeps every cell's density, so the total mass is conserved
    m = o.fluid_totals()[0]
    o.step(20)
    assert abs(o.fluid_totals()[0] - m) < 1e-12 * m


def test_inlet_over_the_whole_periodic_box_is_a_uniform_flow():
    o = oracle.Oracle(6, 5, 7, walls=False, tau=0.8)
    o.set_inlet((0, 6, 0, 5, 0, 7), U)
    o.fluid_init()
    o.step(10)
    f = o.populations().reshape(-1, 19)
    e, w = o.lattice()
    eu = e @ U
    feq = w * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * U @ U)
    assert np.abs(f - feq[None, :]).max() < 1e-15
    assert np.abs(o.velocity().reshape(3, -1) - U[:, None]).max() < 1e-15


def test_empty_inlet_changes_nothing():
    a = oracle.Oracle(6, 8, 6, walls=True, tau=1.0, body_force=(1e-5, 0, 0))
    b = oracle.Oracle(6, 8, 6, walls=True, tau=1.0, body_force=(1e-5, 0, 0))
    b.set_inlet((3, 3, 0, 8, 0, 6), U)   # x0 == x1: no cell
    a.fluid_init()
    b.fluid_init()
    a.step(20)
    b.step(20)
    assert np.array_equal(a.populations(), b.populations())
