"""Pins of the FP64 oracle's membrane part (Sec. 4) and mesh conventions (Sec. 5).

Expected values come from outside the oracle:
  * topology: an independent numpy construction, Euler's formula;
  * angles: textbook dihedral angles of the Platonic solids and planar
    trigonometry of a dented octahedron (a concave edge, theta > pi);
  * stretching and volume forces: central finite differences of the energies
    whose negative gradients they are (ks: E = ks L0 int_1^lambda kappa(m)(m-1) dm
    per edge by Gauss-Legendre quadrature; kv: E = kv (V - V0)^2 / (2 V0));
  * local/global area and volume forces: closed forms on a uniformly scaled
    regular icosahedron;
  * bending: a closed form on an octahedron whose top vertex is moved along
    the axis, zero net force, invariance under uniform scaling, relaxation of
    the angle deviations;
  * measures: scipy's ConvexHull area and volume, the regular icosahedron's
    closed forms, the Evans-Fung closed-form volume;
  * restoration of area and volume after inflation and squashing.
"""
import math

import numpy as np
import pytest
from scipy.spatial import ConvexHull

import oracle
from workloads import mesh


def _sim(nodes, tris, stretch=(1, 1, 1), origin=(0, 0, 0), rotate=(0, 0, 0), nonlinear=1, **k):
    o = oracle.Oracle(64, 64, 64, walls=False)
    tid = o.template_create(nodes, tris, stretch, k.get("ks", 0.0), k.get("kb", 0.0), k.get("kal", 0.0),
                            k.get("kag", 0.0), k.get("kv", 0.0), nonlinear)
    o.object_add(tid, origin, rotate)
    return o


# ----------------------------------------------------------------- topology

@pytest.mark.parametrize("level", [0, 1, 2])
def test_topology_matches_independent_construction(level):
    nodes, tris = mesh.icosphere(level)
    o = _sim(nodes, tris)
    top = o.topology(0, len(tris))
    allpairs = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    uniq = np.unique(allpairs, axis=0)
    assert np.array_equal(top["edges"], uniq.astype(np.int32))
    V, E, F = len(nodes), len(uniq), len(tris)
    assert V - E + F == 2 and E == 3 * F // 2
    cyc = {tuple(np.roll(t, r)) for t in tris.tolist() for r in range(3)}
    for (a, b, c, d), (eb, ec) in zip(top["quads"], top["edges"]):
        assert (b, c) == (eb, ec)
        assert (a, b, c) in cyc and (d, c, b) in cyc and a != d


def test_template_rejects_bad_meshes():
    nodes, tris = mesh.icosphere(1)
    o = oracle.Oracle(8, 8, 8, walls=False)
    with pytest.raises(ValueError):
        o.template_create(nodes, tris[:-1])                  # open mesh
    with pytest.raises(ValueError):
        o.template_create(nodes, tris[:, [0, 2, 1]].copy())  # outward
    bad = tris.copy()
    bad[0] = bad[0][[0, 2, 1]]
    with pytest.raises(ValueError):
        o.template_create(nodes, bad)                        # inconsistent


# ----------------------------------------------------------------- angles

@pytest.mark.parametrize("name,expected", [
    ("tetrahedron", math.acos(1.0 / 3.0)),
    ("octahedron", math.acos(-1.0 / 3.0)),
    ("icosahedron", math.acos(-math.sqrt(5.0) / 3.0)),
])
def test_platonic_inner_dihedral_angles(name, expected):
    nodes, tris = {"tetrahedron": mesh.tetrahedron(), "octahedron": mesh.octahedron(),
                   "icosahedron": mesh.icosphere(0)}[name]
    top = _sim(nodes, tris).topology(0, len(tris))
    assert np.abs(top["theta0"] - expected).max() < 1e-14


def _pyramid_lateral_angle(h):
    # inner angle at a lateral edge of the square pyramid with base
    # (+-1,0,0),(0,+-1,0) and apex height h: outward face normals (h,h,1)
    # and (-h,h,1) make the angle acos(1/(2h^2+1))
    return math.pi - math.acos(1.0 / (2.0 * h * h + 1.0))


def test_dented_octahedron_concave_and_sharp_edges():
    nodes, tris = mesh.octahedron()
    o = _sim(nodes, tris)
    top = o.topology(0, len(tris))
    dented = nodes.copy()
    dented[4] = (0.0, 0.0, -0.5)
    o.object_set_nodes(0, dented)
    th = o.edge_angles(0, len(top["edges"]))
    for (i, j), t in zip(top["edges"], th):
        pair = {int(i), int(j)}
        if 4 in pair:     # spoke of the dent: 2 pi minus the pyramid's angle
            assert abs(t - (2 * math.pi - _pyramid_lateral_angle(0.5))) < 1e-14
            assert t > math.pi
        elif 5 in pair:   # untouched lower spokes
            assert abs(t - math.acos(-1.0 / 3.0)) < 1e-14
        else:             # equator: difference of the two face slopes
            r = math.sqrt(0.5)
            expected = math.atan2(1.0, r) - math.atan2(0.5, r)
            assert abs(t - expected) < 1e-14


# ----------------------------------------------------------------- rest state

def test_all_forces_vanish_at_rest_shape():
    nodes, tris = mesh.biconcave(2)
    o = _sim(nodes, tris, (6, 6, 6), origin=(30.3, 31.7, 29.1), rotate=(0.3, -1.1, 2.0),
             **dict(ks=0.1, kb=0.03, kal=0.1, kag=0.4, kv=1.0))
    for bit in range(5):
        F = o.membrane_forces(0, 1 << bit)
        assert np.abs(F).max() < 1e-12, bit


# ----------------------------------------------------------------- stretching

def _perturbed_sphere(seed=0, level=1, R=3.0, amp=0.05):
    nodes, tris = mesh.icosphere(level)
    rng = np.random.default_rng(seed)
    X = nodes * R + amp * R * rng.standard_normal(nodes.shape) / 3
    return nodes, tris, X


def _gl(n=48):
    return np.polynomial.legendre.leggauss(n)


def _stretch_energy(X, edges, L0, ks, nonlinear):
    d = X[edges[:, 1]] - X[edges[:, 0]]
    lam = np.linalg.norm(d, axis=1) / L0
    if not nonlinear:
        return np.sum(0.5 * ks * L0 * (lam - 1.0) ** 2)
    x, w = _gl()
    mid, half = 0.5 * (lam + 1.0), 0.5 * (lam - 1.0)
    m = mid[:, None] + half[:, None] * x[None, :]
    kap = (m ** 0.5 + m ** -2.5) / (m + m ** -3.0)
    return np.sum(ks * L0 * half * np.sum(w[None, :] * kap * (m - 1.0), axis=1))


def _fd_gradient(energy, X, h=1e-6):
    g = np.zeros_like(X)
    for i in range(X.shape[0]):
        for k in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, k] += h
            Xm[i, k] -= h
            g[i, k] = (energy(Xp) - energy(Xm)) / (2 * h)
    return g


@pytest.mark.parametrize("nonlinear", [1, 0])
def test_stretching_is_minus_gradient_of_energy(nonlinear):
    nodes, tris, X = _perturbed_sphere(1)
    o = _sim(nodes, tris, (3, 3, 3), nonlinear=nonlinear, ks=0.1)
    top = o.topology(0, len(tris))
    o.object_set_nodes(0, X)
    F = o.membrane_forces(0, 1)
    grad = _fd_gradient(lambda Y: _stretch_energy(Y, top["edges"], top["L0"], 0.1, nonlinear), X)
    assert np.abs(F + grad).max() < 1e-7 * np.abs(F).max()
    # symmetric pair forces: no net force
    assert np.abs(F.sum(0)).max() < 1e-15


def test_stretching_known_value_at_lambda_two():
    # One tetrahedron edge (a,b) stretched to twice its length by moving b
    # along it.  The other edges at a keep their rest length, so the force
    # on a along the edge is ks kappa(2) (2 - 1), with
    # kappa(2) = (sqrt 2 + 2^-2.5) / (2 + 2^-3).
    nodes, tris = mesh.tetrahedron()
    o = _sim(nodes, tris, ks=1.0)
    a, b = o.topology(0, len(tris))["edges"][0]
    X = nodes.copy()
    X[b] = X[a] + 2.0 * (X[b] - X[a])
    o.object_set_nodes(0, X)
    F = o.membrane_forces(0, 1)
    d = (X[b] - X[a]) / np.linalg.norm(X[b] - X[a])
    kap2 = (math.sqrt(2.0) + 2.0 ** -2.5) / (2.0 + 0.125)
    assert abs(np.dot(F[a], d) - kap2) < 1e-14


# ----------------------------------------------------------------- volume

def test_volume_force_is_minus_gradient_of_energy():
    nodes, tris, X = _perturbed_sphere(2)
    o = _sim(nodes, tris, (3, 3, 3), kv=1.0)
    V0 = o.topology(0, len(tris))["V0"]
    o.object_set_nodes(0, X)
    F = o.membrane_forces(0, 16)

    def energy(Y):
        o.object_set_nodes(0, Y)
        V = o.object_measures(0)[1]
        return 1.0 * (V - V0) ** 2 / (2 * V0)

    grad = _fd_gradient(energy, X)
    assert np.abs(F + grad).max() < 1e-7 * np.abs(F).max()
    assert np.abs(F.sum(0)).max() < 1e-14


# ----------------------------------------------------------------- areas on an icosahedron

@pytest.mark.parametrize("sigma", [1.1, 0.93])
def test_scaled_icosahedron_area_and_volume_forces_closed_form(sigma):
    nodes, tris = mesh.icosphere(0)          # unit circumradius
    a = 1.0 / math.sin(2 * math.pi / 5)       # edge length
    w_radial = (a / math.sqrt(3.0)) / 1.0     # |P - centroid| / R_c
    ri_over_rc = math.sqrt((5 + 2 * math.sqrt(5)) / 15)
    S_face = math.sqrt(3) / 4 * (a * sigma) ** 2
    r_hat = nodes / np.linalg.norm(nodes, axis=1, keepdims=True)
    for mask, k, expected in [
        (4, dict(kal=0.7), -0.7 * (1 - 1 / sigma ** 2) * 5 * w_radial),
        (8, dict(kag=0.3), -0.3 * (1 - 1 / sigma ** 2) * 5 * w_radial),
        (16, dict(kv=2.0), 2.0 * (sigma ** 3 - 1) * (-5 * S_face / 3 * ri_over_rc)),
    ]:
        o = _sim(nodes, tris, **k)
        o.object_set_nodes(0, nodes * sigma)
        F = o.membrane_forces(0, mask)
        radial = np.einsum("ij,ij->i", F, r_hat)
        tangential = F - radial[:, None] * r_hat
        assert np.abs(radial - expected).max() < 1e-13, mask
        assert np.abs(tangential).max() < 1e-13


def test_icosahedron_measures_closed_form():
    nodes, tris = mesh.icosphere(0)
    a = 1.0 / math.sin(2 * math.pi / 5)
    o = _sim(nodes, tris, (2, 2, 2), origin=(10, 11, 12), rotate=(0.4, 0.2, -0.9))
    Sg, V = o.object_measures(0)
    assert abs(Sg - 5 * math.sqrt(3) * (2 * a) ** 2) < 1e-12
    assert abs(V - 5.0 / 12.0 * (3 + math.sqrt(5)) * (2 * a) ** 3) < 1e-12


@pytest.mark.parametrize("level", [1, 2, 3])
def test_measures_match_convex_hull(level):
    nodes, tris = mesh.icosphere(level)
    o = _sim(nodes, tris, (4, 4, 4), origin=(20.5, 10.25, 9.0), rotate=(1.0, 0.5, 0.25))
    X, _ = o.read_nodes(0)
    hull = ConvexHull(X)
    Sg, V = o.object_measures(0)
    assert abs(Sg - hull.area) < 1e-11 * hull.area
    assert abs(V - hull.volume) < 1e-11 * hull.volume


def test_biconcave_mesh_volume_converges_to_evans_fung():
    ref = mesh.biconcave_volume(8.0)
    errs = []
    for level in (2, 3, 4):
        nodes, tris = mesh.biconcave(level)
        o = _sim(nodes, tris, (8, 8, 8))
        errs.append(abs(o.object_measures(0)[1] - ref) / ref)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3


# ----------------------------------------------------------------- bending

def test_bending_closed_form_on_raised_octahedron():
    nodes, tris = mesh.octahedron()
    kb = 0.8
    h = 1.3
    o = _sim(nodes, tris, kb=kb)
    X = nodes.copy()
    X[4] = (0.0, 0.0, h)
    o.object_set_nodes(0, X)
    F = o.membrane_forces(0, 2)
    th0 = math.acos(-1.0 / 3.0)
    th_spoke = _pyramid_lateral_angle(h)
    r = math.sqrt(0.5)
    th_eq = math.atan2(h, r) + math.atan2(1.0, r)
    s_spoke = kb * (th_spoke - th0) / th0
    s_eq = kb * (th_eq - th0) / th0
    # inward unit normals: top faces -(h,h,1)/sqrt(2h^2+1), bottom faces
    # (-1,-1,1)/sqrt(3) up to sign of x,y; only z survives on the axis
    top_z = 4.0 * (s_spoke - s_eq) / math.sqrt(2 * h * h + 1)
    bottom_z = 4.0 * s_eq / math.sqrt(3.0)
    assert np.abs(F[4] - [0, 0, top_z]).max() < 1e-14
    assert np.abs(F[5] - [0, 0, bottom_z]).max() < 1e-14
    assert np.abs(F.sum(0)).max() < 1e-14


def test_bending_zero_net_force_and_scale_invariance():
    nodes, tris, X = _perturbed_sphere(3, level=2)
    o = _sim(nodes, tris, (3, 3, 3), kb=0.03)
    o.object_set_nodes(0, X)
    F = o.membrane_forces(0, 2)
    assert np.abs(F).max() > 1e-5
    assert np.abs(F.sum(0)).max() < 1e-15
    o.object_set_nodes(0, nodes * 3 * 1.37)
    assert np.abs(o.membrane_forces(0, 2)).max() < 1e-13


def test_bending_relaxes_angle_deviation():
    nodes, tris, X = _perturbed_sphere(4, level=1, amp=0.04)
    o = _sim(nodes, tris, (3, 3, 3), kb=0.5)
    top = o.topology(0, len(tris))
    ne = len(top["edges"])
    o.object_set_nodes(0, X)
    dev0 = np.abs(o.edge_angles(0, ne) - top["theta0"]).max()
    Y = X.copy()
    for _ in range(400):
        Y = Y + 0.05 * o.membrane_forces(0, 2)
        o.object_set_nodes(0, Y)
    dev1 = np.abs(o.edge_angles(0, ne) - top["theta0"]).max()
    assert dev1 < 0.1 * dev0


# ----------------------------------------------------------------- restoration

@pytest.mark.parametrize("deform", ["inflate", "squash"])
def test_area_and_volume_restored_after_deformation(deform):
    nodes, tris = mesh.icosphere(2)
    o = _sim(nodes, tris, (4, 4, 4), origin=(32, 32, 32), ks=0.1, kb=0.03, kal=0.1, kag=0.4, kv=1.0)
    top = o.topology(0, len(tris))
    X0, _ = o.read_nodes(0)
    c = X0.mean(0)
    X = c + (X0 - c) * (1.1 if deform == "inflate" else np.array([1.0, 1.0, 0.8]))
    o.object_set_nodes(0, X)
    Sg, V = o.object_measures(0)
    assert abs(V / top["V0"] - 1) > 0.05
    for _ in range(3000):
        X = X + 0.1 * o.membrane_forces(0, 31)
        o.object_set_nodes(0, X)
    Sg, V = o.object_measures(0)
    assert abs(Sg / top["Sg0"] - 1) < 1e-3
    assert abs(V / top["V0"] - 1) < 1e-3


# ----------------------------------------------------------------- placement

def test_rotation_order_and_translation():
    nodes, tris = mesh.tetrahedron()
    o = _sim(nodes, tris, origin=(1.0, 2.0, 3.0), rotate=(math.pi / 2, 0.0, 0.0))
    X, _ = o.read_nodes(0)
    # about x by +90 degrees: (x, y, z) -> (x, -z, y)
    exp = np.stack([nodes[:, 0], -nodes[:, 2], nodes[:, 1]], 1) + [1, 2, 3]
    assert np.abs(X - exp).max() < 1e-15
    o2 = _sim(nodes, tris, rotate=(math.pi / 2, math.pi / 2, 0.0))
    X2, _ = o2.read_nodes(0)
    # x first: (x,y,z)->(x,-z,y); then y by 90: (x,y,z)->(z,y,-x)
    step1 = np.stack([nodes[:, 0], -nodes[:, 2], nodes[:, 1]], 1)
    exp2 = np.stack([step1[:, 2], step1[:, 1], -step1[:, 0]], 1)
    assert np.abs(X2 - exp2).max() < 1e-15


def test_local_area_along_altitudes_is_the_normalised_area_gradient():
    """Second direction of Sec. 4 for the local-area force: along each
    vertex's altitude.  That direction is the direction of the gradient of
    the triangle's area with respect to the vertex, taken here by central
    finite differences of the area, an independent route."""
    nodes, tris = mesh.icosphere(0)
    o = oracle.Oracle(20, 20, 20, walls=False)
    o.template_create(nodes, tris, (3.0, 2.0, 1.5), kal=0.1)   # stretched: non-equilateral triangles
    o.template_set_kal_direction(0, True)
    o.object_add(0, (10.0, 10.0, 10.0))
    X0, _ = o.read_nodes(0)
    rng = np.random.default_rng(3)
    X = X0 + rng.normal(0.0, 0.05, X0.shape)
    o.object_set_nodes(0, X)
    F = o.membrane_forces(0, 4)
    area = lambda a, b, c: 0.5 * np.linalg.norm(np.cross(b - a, c - a))  # noqa: E731
    S0 = [area(*X0[t]) for t in tris]
    exp = np.zeros_like(X)
    h = 1e-6
    for t, s0 in zip(tris, S0):
        P = X[t].copy()
        S = area(*P)
        for j in range(3):
            g = np.zeros(3)
            for k in range(3):
                Pp, Pm = P.copy(), P.copy()
                Pp[j, k] += h
                Pm[j, k] -= h
                g[k] = (area(*Pp) - area(*Pm)) / (2 * h)
            exp[t[j]] += -0.1 * (S - s0) / S * g / np.linalg.norm(g)
    assert np.abs(F - exp).max() < 1e-8 * np.abs(exp).max()


def test_local_area_directions_agree_on_equilateral_faces():
    nodes, tris = mesh.icosphere(0)   # regular icosahedron: every face equilateral
    out = []
    for alt in (False, True):
        o = oracle.Oracle(20, 20, 20, walls=False)
        o.template_create(nodes, tris, (2.0, 2.0, 2.0), kal=0.1)
        o.template_set_kal_direction(0, alt)
        o.object_add(0, (10.0, 10.0, 10.0))
        X0, _ = o.read_nodes(0)
        o.object_set_nodes(0, 10.0 + (X0 - 10.0) * 1.1)   # uniform inflation keeps faces equilateral
        out.append(o.membrane_forces(0, 4))
    assert np.abs(out[1]).max() > 0
    assert np.allclose(out[0], out[1], rtol=1e-12, atol=1e-15)
