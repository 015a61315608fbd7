"""The allocation-free mass reduction (lbib_fluid_mass_noalloc) against the
allocating one (lbib_fluid_mass) on the same state, two calls in a row.
Collected last on purpose: it must also pass after every other GPU test has
used the device."""
import numpy as np
import pytest

from paper_1312_3426_gb300 import lbib
from workloads import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_3426_gb300 import build
    build.build()
    lbib.load()


@pytest.mark.parametrize("prec,scale", [("f32", 0), ("f16s", 12)])
def test_noalloc_mass_equals_allocating_mass(prec, scale):
    sc = scenes.channel_sphere()
    g = lbib.Sim.from_scene(sc, precision=prec, pop_scale_log2=scale)
    g.step(60)
    for _ in range(2):  # two calls in a row on the same state
        a = lbib.lbib_fluid_mass(g.h)
        b1 = lbib.lbib_fluid_mass_noalloc(g.h)
        b2 = lbib.lbib_fluid_mass_noalloc(g.h)
        assert b1 == b2                       # fixed summation order: deterministic
        assert abs(a - b1) <= 1e-12 * abs(a)  # FP64 sums differing only in order
    g.step(7)
    assert abs(lbib.lbib_fluid_mass(g.h) - lbib.lbib_fluid_mass_noalloc(g.h)) <= 1e-12 * abs(a)
    # a second simulation on the same device uses the same scratch afterwards
    h = lbib.Sim.from_scene(scenes.channel_sphere(with_object=False))
    h.step(5)
    m = lbib.lbib_fluid_mass_noalloc(h.h)
    assert m == pytest.approx(lbib.lbib_fluid_mass(h.h), rel=1e-12)
    assert np.isfinite(m)
    g.close()
    h.close()
