"""Values the paper prints, read from tests/golden/ (each line cites its
section), against the inputs the oracle and the library are run on.

The drag reading rests on these numbers: the example couples the objects
with friction 0.5 at an integration time step of 0.1, so one lattice step
(the library's unit time step) exchanges 0.5 x 0.1 = 0.05 of the relative
velocity for a unit-mass node; the scenes use xi = 0.05 per step."""
import os

import pytest

from workloads import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_example_parameters.txt")) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            name, value, src = ln.split()
            vals[name] = (float(value), src)
    return vals


def test_moduli_are_the_papers():
    g = _golden()
    for k in ("ks", "kb", "kal", "kag", "kv"):
        assert scenes.PAPER_MODULI[k] == g[k][0], k


def test_drag_per_lattice_step_is_friction_times_time_step():
    g = _golden()
    assert scenes.Scene("x", 4, 4, 4).friction == pytest.approx(g["friction"][0] * g["md_time_step"][0])
    assert g["lb_tau"][0] == g["md_time_step"][0]  # one object update per fluid step


def test_node_mass_default_is_unit():
    g = _golden()
    assert scenes.Obj(0, (0, 0, 0)).mass == g["node_mass"][0]


def test_repulsion_in_lattice_units_is_the_papers_times_time_step_squared():
    g = _golden()
    dt2 = g["md_time_step"][0] ** 2
    (oa, on, orc), (wa, wn, wrc) = scenes.PAPER_REPULSION
    assert oa == pytest.approx(g["soft_obj_a"][0] * dt2) and on == g["soft_obj_n"][0]
    assert orc == g["soft_obj_cutoff"][0]
    assert wa == pytest.approx(g["soft_wall_a"][0] * dt2) and wn == g["soft_wall_n"][0]
    assert wrc == g["soft_wall_cutoff"][0]
