"""Failure detection without a GPU fault: the device-side waits of the
warp-specialised fluid kernel are bounded by the global timer.  A kernel
waits on a shared-memory barrier that nothing completes; the wait must give
up after its bound, report the timeout to the host through a status word,
and leave the context usable for the next simulation."""
import time

import numpy as np
import pytest

from paper_1312_3426_gb300 import lbib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_3426_gb300 import build
    build.build()
    lbib.load()


def test_wait_on_a_barrier_nothing_completes_times_out():
    t0 = time.perf_counter()
    assert lbib.lbib_check_bounded_wait(0.2, arrive=False)
    dt = time.perf_counter() - t0
    assert 0.2 <= dt < 5.0, dt


def test_wait_on_a_completed_barrier_does_not_time_out():
    t0 = time.perf_counter()
    assert not lbib.lbib_check_bounded_wait(0.2, arrive=True)
    assert time.perf_counter() - t0 < 5.0


def test_context_usable_after_a_timeout():
    assert lbib.lbib_check_bounded_wait(0.1, arrive=False)
    g = lbib.Sim(24, 12, 16, walls=True, tau=0.8, rho0=1.0, body_force=(1e-5, 0.0, 0.0), friction=0.5)
    g.fluid_init()
    m0 = g.mass()
    g.step(50)
    u = g.velocity()
    m1 = g.mass()
    g.close()
    assert np.isfinite(u).all()
    assert u[0][:, 1:11, :].min() > 0.0  # the body force drives +x flow between the walls
    assert abs(m1 - m0) / m0 < 1e-6
