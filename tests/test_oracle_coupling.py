"""Pins of the FP64 oracle's fluid-object coupling (Sec. 2, Eq. dragforce, Eq. newton).

  * interpolation reproduces the value at a lattice node and any linear field;
  * spreading uses the cuboid-volume weights computed here from their
    definition, and the fluid receives exactly minus the drag;
  * a node at rest in a frozen uniform flow U reaches v_k = U (1 - (1 - xi/m)^k);
  * in a fully periodic box the total momentum of fluid plus nodes is
    conserved when only momentum-free moduli (ks, kb, kv) are on;
  * solid corners contribute u = 0 and the momentum they would receive is
    recorded as dropped.
"""
import itertools

import numpy as np

import oracle
from workloads import mesh


def _frozen(nx=12, ny=12, nz=12, walls=False, xi=0.5):
    o = oracle.Oracle(nx, ny, nz, walls=walls, friction=xi)
    o.fluid_init()
    return o


def test_interpolation_exact_at_node_and_for_linear_fields():
    o = _frozen()
    rng = np.random.default_rng(0)
    u = rng.standard_normal((3, 12, 12, 12))
    o.set_velocity(u)
    for (i, j, k) in [(3, 4, 5), (0, 0, 0), (7, 2, 9)]:
        got = o.interpolate([i + 0.5, j + 0.5, k + 0.5])
        assert np.abs(got - u[:, k, j, i]).max() == 0.0
    A = rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    zz, yy, xx = np.meshgrid(np.arange(12) + 0.5, np.arange(12) + 0.5, np.arange(12) + 0.5, indexing="ij")
    pos = np.stack([xx, yy, zz])
    lin = np.einsum("ab,bzyx->azyx", A, pos) + b[:, None, None, None]
    o.set_velocity(lin)
    for _ in range(20):
        X = 1.0 + 9.0 * rng.random(3)
        assert np.abs(o.interpolate(X) - (A @ X + b)).max() < 1e-13


def _cuboid_weights(X):
    """Weight of each of the 8 surrounding nodes: the volume of the box
    between X and the node diagonally opposite to it."""
    lo = np.floor(X - 0.5).astype(int)
    out = {}
    for d in itertools.product((0, 1), repeat=3):
        node = lo + np.array(d)
        opposite = lo + 1 - np.array(d)
        centre_opp = opposite + 0.5
        out[tuple(node)] = float(np.prod(np.abs(X - centre_opp)))
    return out


def test_spreading_weights_and_sum_equal_minus_drag():
    o = _frozen(xi=0.7)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((3, 12, 12, 12)) * 1e-2
    o.set_velocity(U)
    nodes, tris = mesh.tetrahedron()
    tid = o.template_create(nodes, tris, (0.3, 0.3, 0.3))
    o.object_add(tid, (5.37, 6.11, 4.83))
    X, V = o.read_nodes(0)
    drag = np.array([0.7 * (o.interpolate(x) - v) for x, v in zip(X, V)])
    o.step_nodes_only(1)
    G = o.ib_force()
    expected = np.zeros_like(G)
    for x, fd in zip(X, drag):
        for (i, j, k), w in _cuboid_weights(x).items():
            expected[:, k % 12, j % 12, i % 12] -= w * fd
    assert np.abs(G - expected).max() < 1e-16
    assert np.abs(G.reshape(3, -1).sum(1) + drag.sum(0)).max() < 1e-16


def test_node_relaxes_geometrically_to_frozen_uniform_flow():
    xi, m = 0.5, 2.0
    o = _frozen(xi=xi)
    U = np.array([3e-3, -1e-3, 2e-3])
    o.set_velocity(np.broadcast_to(U[:, None, None, None], (3, 12, 12, 12)).copy())
    nodes, tris = mesh.tetrahedron()
    tid = o.template_create(nodes, tris, (0.5, 0.5, 0.5))
    o.object_add(tid, (6.0, 6.0, 6.0), mass=m)
    for k in range(1, 9):
        o.step_nodes_only(1)
        _, V = o.read_nodes(0)
        expected = U * (1.0 - (1.0 - xi / m) ** k)
        assert np.abs(V - expected).max() < 1e-17


def test_external_force_accelerates_free_object():
    o = _frozen(xi=0.0)
    nodes, tris = mesh.tetrahedron()
    tid = o.template_create(nodes, tris)
    o.object_add(tid, (6.0, 6.0, 6.0), mass=4.0)
    o.object_set_force(0, (1e-3, 0.0, -2e-3))
    X0, _ = o.read_nodes(0)
    o.step_nodes_only(3)
    X, V = o.read_nodes(0)
    a = np.array([1e-3, 0.0, -2e-3]) / 4.0
    assert np.abs(V - 3 * a).max() < 1e-18
    # symplectic Euler: X_k = X_0 + a (1 + 2 + ... + k)
    assert np.abs(X - X0 - 6 * a).max() < 1e-15


def test_total_momentum_conserved_fluid_plus_nodes_periodic():
    o = oracle.Oracle(14, 14, 14, walls=False, tau=0.9, friction=0.5)
    o.fluid_init()
    nodes, tris = mesh.icosphere(1)
    tid = o.template_create(nodes, tris, (3, 3, 3), ks=0.1, kb=0.03, kal=0.0, kag=0.0, kv=1.0)
    o.object_add(tid, (7.1, 6.8, 7.3), rotate=(0.2, 0.4, 0.1), mass=1.5)
    rng = np.random.default_rng(5)
    X, _ = o.read_nodes(0)
    o.object_set_nodes(0, X + 0.1 * rng.standard_normal(X.shape))
    V0 = 1e-3 * rng.standard_normal(X.shape)
    o.object_set_velocities(0, V0)
    f = o.populations()
    o.set_populations(f * (1 + 1e-3 * rng.standard_normal(f.shape)))

    def total():
        _, p = o.fluid_totals()
        _, v = o.read_nodes(0)
        return p + 1.5 * v.sum(0)

    p0 = total()
    o.step(60)
    p1 = total()
    assert np.abs(p1 - p0).max() < 1e-13
    assert np.abs(o.dropped()).max() == 0.0


def test_solid_corners_give_zero_velocity_and_drop_force():
    o = oracle.Oracle(10, 10, 10, walls=True, friction=0.5)
    o.fluid_init()
    u = np.ones((3, 10, 10, 10)) * 1e-2
    o.set_velocity(u)
    # y = 1.2: corners in rows 0 (solid, weight 0.3) and 1 (fluid, weight 0.7)
    got = o.interpolate([4.5, 1.2, 4.5])
    assert np.abs(got - 0.7e-2).max() < 1e-17
    nodes, tris = mesh.tetrahedron()
    tid = o.template_create(nodes, tris, (1e-3, 1e-3, 1e-3))
    o.object_add(tid, (4.5, 1.2, 4.5))
    o.step_nodes_only(1)
    G = o.ib_force()
    assert np.abs(G[:, :, 0, :]).max() == 0.0
    total = G.reshape(3, -1).sum(1) + o.dropped()
    X, V = o.read_nodes(0)
    assert np.abs(total + 4 * 0.5 * 0.7e-2).max() < 1e-15
