"""Pins of the FP64 oracle's fluid part against what the mathematics fixes.

Nothing here compares the oracle with itself: every expected value is a
closed form, a lattice identity or a conservation law.
  * D3Q19 weights: the moment identities that define the lattice (Sec. 2).
  * Eq. lbequation: mass and momentum conservation of the
    collision (Sec. 2, the operator conserves both), equilibrium at rest,
    the exact momentum gain G per step under a uniform force, and the
    velocity (t - 1/2) G / rho of the half-force definition.
  * Poiseuille flow between halfway bounce-back walls: the steady BGK
    solution is the parabola u(y) = g/(2 nu) (y-1)(ny-1-y) plus a constant
    slip g (16 L - 3)/(24 nu), L = (tau-1/2)^2.  At the "magic" value
    L = 3/16 (tau = 1/2 + sqrt(3)/4) the slip vanishes and the parabola is
    exact (the standard TRT/BGK bounce-back result).
"""
import math

import numpy as np
import pytest

import oracle


def _box(nx, ny, nz, walls=True, tau=1.0, g=(0, 0, 0)):
    o = oracle.Oracle(nx, ny, nz, walls=walls, tau=tau, rho0=1.0, body_force=g, friction=0.5)
    o.fluid_init()
    return o


def test_d3q19_moment_identities():
    e, w = _box(2, 3, 2).lattice()
    e = e.astype(np.float64)
    assert len(w) == 19
    assert len({tuple(v) for v in e.astype(int)}) == 19
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-16
    second = np.einsum("q,qa,qb->ab", w, e, e)
    assert np.abs(second - np.eye(3) / 3.0).max() < 1e-15
    fourth = np.einsum("q,qa,qb,qc,qd->abcd", w, e, e, e, e)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.abs(fourth - iso).max() < 1e-15
    # every direction has its opposite
    for v in e:
        assert any(np.array_equal(-v, u) for u in e)


def test_equilibrium_at_rest_is_invariant():
    o = _box(6, 8, 5)
    f0 = o.populations().copy()
    o.step(50)
    f = o.populations()
    fluid = np.ones(f.shape[:3], bool)
    fluid[:, 0] = fluid[:, -1] = False
    assert np.abs(f[fluid] - f0[fluid]).max() < 1e-15
    assert np.abs(o.velocity()).max() < 1e-15


def _random_state(o, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    f = o.populations()
    f = f * (1.0 + amp * rng.standard_normal(f.shape))
    o.set_populations(f)
    return f


def test_collision_and_streaming_conserve_mass_and_momentum_periodic():
    o = _box(5, 4, 6, walls=False)
    _random_state(o, 0)
    m0, p0 = o.fluid_totals()
    o.step(40)
    m1, p1 = o.fluid_totals()
    assert abs(m1 - m0) / m0 < 1e-14
    assert np.abs(p1 - p0).max() < 1e-14


def test_mass_conserved_with_walls():
    o = _box(6, 9, 5, walls=True, g=(1e-4, 0, 0))
    _random_state(o, 1)
    m0, _ = o.fluid_totals()
    o.step(300)
    m1, _ = o.fluid_totals()
    assert abs(m1 - m0) / m0 < 1e-13


def test_uniform_force_momentum_gain_and_half_force_velocity():
    g = np.array([2e-5, -1e-5, 3e-6])
    o = _box(4, 3, 5, walls=False, g=g)
    ncell = 4 * 3 * 5
    for t in range(1, 6):
        _, p_before = o.fluid_totals()
        o.step(1)
        _, p_after = o.fluid_totals()
        assert np.allclose(p_after - p_before, ncell * g, rtol=0, atol=1e-14)
        u = o.velocity().reshape(3, -1)
        # u at step t = (sum f e + G/2)/rho with sum f e = (t-1) G, rho = 1
        assert np.abs(u - ((t - 0.5) * g)[:, None]).max() < 1e-16


def _poiseuille(tau, ny=20, g=1e-5, steps=None):
    nu = (tau - 0.5) / 3.0
    H = ny - 2
    if steps is None:
        steps = int(40 * H * H / (math.pi ** 2 * nu)) + 200
    o = _box(2, ny, 2, walls=True, tau=tau, g=(g, 0, 0))
    o.step(steps)
    u = o.velocity()[0, 0, :, 0]
    y = np.arange(ny) + 0.5
    parabola = g / (2 * nu) * (y - 1.0) * (ny - 1.0 - y)
    slip = g * (16.0 * (tau - 0.5) ** 2 - 3.0) / (24.0 * nu)
    return u[1:-1], parabola[1:-1], slip


@pytest.mark.parametrize("tau", [1.0, 0.8, 0.5 + math.sqrt(3) / 4, 1.4])
def test_poiseuille_parabola_plus_slip(tau):
    u, par, slip = _poiseuille(tau)
    err = np.abs(u - (par + slip)).max() / par.max()
    assert err < 1e-10, err


def test_poiseuille_magic_tau_has_no_slip():
    u, par, slip = _poiseuille(0.5 + math.sqrt(3) / 4)
    assert abs(slip) < 1e-18
    assert np.abs(u - par).max() / par.max() < 1e-10


def test_poiseuille_profile_tau1_matches_quoted_error():
    # relative L2 distance of the steady tau=1 profile to the bare parabola,
    # a consequence of the slip alone (H = 18)
    u, par, _ = _poiseuille(1.0)
    rel = np.linalg.norm(u - par) / np.linalg.norm(par)
    assert 1.3e-3 < rel < 1.5e-3


def test_channel_is_invariant_along_x_and_z_and_symmetric():
    u, _, _ = _poiseuille(1.0, steps=400)
    assert np.abs(u - u[::-1]).max() < 1e-16


def test_density_readout_uniform_in_driven_channel_and_mass_of_the_box():
    """The steady body-force-driven channel has a uniform pressure, so the
    density read-out is rho0 in every fluid cell (Eq. lbequation: the force
    adds no mass); at rest after initialisation it is rho0 too; and the
    read-out sums to the conserved total over the fluid cells."""
    o = _box(3, 12, 2, walls=True, tau=0.9, g=(1e-5, 0, 0))
    rho = o.density()
    assert np.abs(rho[:, 1:-1, :] - 1.0).max() == 0.0
    o.step(3000)
    rho = o.density()[:, 1:-1, :]
    assert np.abs(rho - 1.0).max() < 1e-12
    assert abs(rho.sum() - o.fluid_totals()[0]) < 1e-10
    assert abs(rho.sum() - 3 * 10 * 2) < 1e-10
