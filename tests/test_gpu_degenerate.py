"""Degenerate boxes: dimensions one or two cells wide (every neighbour is the
cell itself or its one partner through the periodic wrap), a single fluid
row between the walls, a single fully periodic cell, and zero steps.  Each
is run object-free with a body force on the GPU (FP32 and FP16-shifted
storage; the two-cells kernel where nx is even) and compared with the FP64
oracle on the same box.  The single periodic cell also has a closed form:
every step adds the force to the momentum, and the velocity of the last
collision carries half the force of that step, so after t steps
u = F (t - 1/2) / rho0 exactly in exact arithmetic.  Total mass: FP32
storage within 1e-6 relative; FP16-shifted storage within six standard
deviations of the random walk its unbiased stochastic rounding makes.
"""
import numpy as np
import pytest

import oracle
from paper_1312_3426_gb300 import lbib

pytestmark = pytest.mark.gpu

FORCE = (1e-5, 2e-6, -3e-6)
STEPS = 300
BOXES = [  # nx, ny, nz, walls
    (1, 1, 1, False),
    (1, 3, 1, True),
    (2, 5, 1, True),
    (1, 20, 7, True),
    (64, 3, 2, True),
    (3, 4, 5, False),
    (2, 2, 2, False),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_3426_gb300 import build
    build.build()
    lbib.load()


def rel(a, b):
    n = float(np.linalg.norm(b))
    return float(np.linalg.norm(a.astype(np.float64) - b)) / n


@pytest.mark.parametrize("prec,scale,bound", [("f32", 0, 1e-5), ("f16s", 12, 5e-3)])
@pytest.mark.parametrize("nx,ny,nz,walls", BOXES)
def test_degenerate_box_matches_oracle(nx, ny, nz, walls, prec, scale, bound):
    force = FORCE if not walls else (FORCE[0], 0.0, FORCE[2])  # no force into a wall
    o = oracle.Oracle(nx, ny, nz, walls=walls, tau=0.8, rho0=1.0, body_force=force, friction=0.5)
    o.fluid_init()
    o.step(STEPS)
    g = lbib.Sim(nx, ny, nz, walls=walls, tau=0.8, rho0=1.0, body_force=force, friction=0.5,
                 precision=prec, pop_scale_log2=scale)
    g.fluid_init()
    g.step(STEPS)
    ug = g.velocity()
    m = g.mass()
    hmax = float(np.abs(g.populations()).max())
    g.close()
    uo = o.velocity()
    rows = slice(1, ny - 1) if walls else slice(0, ny)
    err = rel(ug[:, :, rows, :], uo[:, :, rows, :])
    print(f"\n{nx}x{ny}x{nz} walls={walls} {prec}: relative L2 {err:.3e}")
    assert err <= bound, err
    nfluid = nx * (ny - 2 if walls else ny) * nz
    if prec == "f32":
        assert abs(m - nfluid) <= 1e-6 * nfluid
    else:
        # Stochastic rounding is unbiased: the mass walks by independent
        # zero-mean errors, one per stored number and step, each smaller than
        # one ulp of that number (standard deviation at most half an ulp), so
        # in a box this small it is bounded statistically, not to 1e-6.
        ulp = 2.0 ** (np.floor(np.log2(hmax * 2 ** scale)) - 10) / 2 ** scale
        assert abs(m - nfluid) <= 6 * 0.5 * ulp * np.sqrt(STEPS * 19 * nfluid)


def test_single_periodic_cell_closed_form():
    g = lbib.Sim(1, 1, 1, walls=False, tau=0.8, rho0=1.0, body_force=FORCE, friction=0.5)
    g.fluid_init()
    g.step(STEPS)
    u = g.velocity()[:, 0, 0, 0].astype(np.float64)
    g.close()
    exact = np.array(FORCE) * (STEPS - 0.5)
    assert np.abs(u - exact).max() <= 1e-5 * np.abs(exact).max(), (u, exact)


def test_zero_steps_change_nothing():
    g = lbib.Sim(16, 10, 8, walls=True, tau=1.0, rho0=1.0, body_force=(1e-5, 0.0, 0.0), friction=0.5)
    g.fluid_init()
    p0 = g.populations()
    g.step(0)
    g.sync()
    assert np.abs(g.velocity()).max() == 0.0
    assert np.array_equal(g.populations(), p0)
    g.close()
