"""The allocation-free mass reduction (lbib_fluid_mass_noalloc): exact at
rest, equal to the FP64 oracle's total after stepping (with and without
obstacle cells), equal to the allocating lbib_fluid_mass on the same state
on two calls in a row, and without any device allocation.
Collected last on purpose: it must also pass after every other GPU test has
used the device."""
import numpy as np
import pytest

import oracle
from paper_1312_3426_gb300 import lbib
from workloads import geometry, mesh, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_3426_gb300 import build
    build.build()
    lbib.load()


def _obstacle_scene():
    s = scenes.Scene("posts", 40, 16, 24, walls=True, body_force=(2e-5, 0.0, 0.0))
    s.solid = geometry.staggered_rhomboids(40, 16, 24, count=3, seed=5)
    n2, t2 = mesh.biconcave(2)
    s.templates.append(scenes.Template(n2, t2, (3.0, 3.0, 3.0), **scenes.PAPER_MODULI))
    s.objects.append(scenes.Obj(0, (20.0, 8.0, 4.5), (0.3, 0.2, 0.1)))
    return s


def _fluid_cells(sc):
    """Cells that hold fluid: the rows between the walls minus obstacles."""
    rows = slice(1, sc.ny - 1) if sc.walls else slice(0, sc.ny)
    n = sc.nx * (sc.ny - 2 if sc.walls else sc.ny) * sc.nz
    solid = getattr(sc, "solid", None)
    return n - (int(np.count_nonzero(solid[:, rows, :])) if solid is not None else 0)


@pytest.mark.parametrize("prec,scale", [("f32", 0), ("f16s", 12), ("bf16s", 12)])
@pytest.mark.parametrize("which", ["sphere", "obstacles"])
def test_noalloc_mass_is_exact_at_rest(prec, scale, which):
    """Right after lbib_fluid_init every deviation is zero, so the total is
    (fluid cells) x rho0 exactly."""
    sc = scenes.channel_sphere() if which == "sphere" else _obstacle_scene()
    g = lbib.Sim.from_scene(sc, precision=prec, pop_scale_log2=scale)
    assert lbib.lbib_fluid_mass_noalloc(g.h) == _fluid_cells(sc) * sc.rho0
    g.close()


@pytest.mark.parametrize("which", ["sphere", "obstacles"])
def test_noalloc_mass_matches_oracle(which):
    """After stepping, the FP32 path's total against the FP64 oracle's
    (the deviations are summed in FP64; the difference is the FP32
    rounding of the collisions)."""
    sc = scenes.channel_sphere() if which == "sphere" else _obstacle_scene()
    o = oracle.Oracle.from_scene(sc)
    g = lbib.Sim.from_scene(sc)
    o.step(200)
    g.step(200)
    m_o = o.fluid_totals()[0]
    m = lbib.lbib_fluid_mass_noalloc(g.h)
    assert abs(m - m_o) <= 1e-9 * m_o, (m, m_o)
    g.close()


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


def test_noalloc_mass_allocates_nothing():
    """Free device memory and the simulation's held bytes stay the same
    over repeated calls (after a first call has loaded the kernel)."""
    torch = pytest.importorskip("torch")
    g = lbib.Sim.from_scene(scenes.channel_sphere())
    g.step(10)
    lbib.lbib_fluid_mass_noalloc(g.h)
    free0, _ = torch.cuda.mem_get_info()
    held0 = g.info()[5]
    vals = [lbib.lbib_fluid_mass_noalloc(g.h) for _ in range(20)]
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and g.info()[5] == held0
    assert len(set(vals)) == 1
    g.close()
