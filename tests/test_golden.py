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


def _channel_profile():
    import numpy as np
    return np.loadtxt(os.path.join(HERE, "golden", "channel_512x256x256_profile.txt"))


def test_channel_profile_file_is_the_oracles():
    """The stored 512x256x256 channel profile (the bench's Poiseuille
    reference) is what the oracle computes (written by
    tests/golden/make_channel_profile.py)."""
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_channel_profile
    u = make_channel_profile.profile()
    assert (u == _channel_profile()).all()


def test_channel_profile_against_the_start_up_series():
    """Independent of the oracle: the continuum start-up of plane Poiseuille
    flow between the halfway walls y = 1 and y = 255 (H = 254, nu = 1/6,
    g = 1e-5, BGK slip u_s = g (16 (tau - 1/2)^2 - 3) / (24 nu)),
    u(s, t) = u_ss(s) - sum_{n odd} 4 g H^2 / (nu pi^3 n^3)
    sin(n pi s / H) exp(-nu n^2 pi^2 t / H^2), at the cell centres
    s = y - 1/2, t = 20,000; walls have u = 0.  The lattice solution agrees
    to the lattice's discretisation error."""
    import numpy as np
    u = _channel_profile()
    g, nu, H, t, tau = 1e-5, 1.0 / 6.0, 254.0, 20000.0, 1.0
    s = np.arange(1, 255) - 0.5
    us = g * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu)
    series = g / (2 * nu) * s * (H - s) + us
    for n in range(1, 400, 2):
        series -= 4 * g * H ** 2 / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * s / H) * \
            np.exp(-nu * n ** 2 * np.pi ** 2 * t / H ** 2)
    err = np.linalg.norm(u[1:255] - series) / np.linalg.norm(series)
    assert err < 1e-4, err  # measured 2.9e-5
    assert u[0] == 0.0 and u[255] == 0.0
    assert np.abs(u[1:255] - u[254:0:-1]).max() <= 1e-15  # symmetric about the centre
