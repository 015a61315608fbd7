"""C-ABI checks that need no GPU: the library loads, exports every entry
point declared in include/lbib.h, its D3Q19 table is the lattice of Sec. 2,
and its host-side mesh builder gives bit-exactly the oracle's brute-force
topology (edges, bending quadruples) with matching relaxed measures."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1312_3426_gb300 import lbib
from workloads import mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbib.h")).read()
    return sorted(set(re.findall(r"LBIB_API\s+[\w\s\*]*?\b(lbib_\w+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    lib = lbib.load()
    names = _declared_symbols()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert lbib.lbib_abi_version() == 1


def test_lattice_is_d3q19_and_matches_oracle_set():
    e, w = lbib.lbib_lattice()
    eo, wo = oracle.Oracle(2, 3, 2).lattice()
    assert {(tuple(a), b) for a, b in zip(e.tolist(), w.tolist())} == \
           {(tuple(a), b) for a, b in zip(eo.tolist(), wo.tolist())}
    assert e[0].tolist() == [0, 0, 0]
    for q in range(1, 19):   # opposite of q is q+1 (odd q) / q-1 (even q)
        opp = q + 1 if q % 2 else q - 1
        assert (e[opp] == -e[q]).all()


def _meshes():
    yield "ico0", mesh.icosphere(0), (1, 1, 1)
    yield "ico2", mesh.icosphere(2), (4, 4, 4)
    yield "ico3", mesh.icosphere(3), (4, 4, 4)
    yield "rbc2", mesh.biconcave(2), (8, 8, 8)
    yield "rbc3", mesh.biconcave(3), (8, 8, 8)
    yield "tet", mesh.tetrahedron(), (1, 2, 3)
    yield "oct", mesh.octahedron(), (1, 1, 1)


@pytest.mark.parametrize("name,nt,stretch", [(n, m, s) for n, m, s in _meshes()])
def test_topology_bit_exact_against_oracle(name, nt, stretch):
    nodes, tris = nt
    lib = lbib.lbib_mesh_check(nodes, tris, stretch)
    o = oracle.Oracle(4, 4, 4, walls=False)
    o.template_create(nodes, tris, stretch)
    ref = o.topology(0, len(tris))
    assert np.array_equal(lib["edges"], ref["edges"])
    assert np.array_equal(lib["quads"], ref["quads"])
    # the device's per-edge record holds edge e's stretching and bending:
    # edge e must be the middle pair (b, c) of quad e
    assert np.array_equal(lib["quads"][:, 1:3], lib["edges"])
    assert np.allclose(lib["L0"], ref["L0"], rtol=1e-14, atol=0)
    assert np.allclose(lib["theta0"], ref["theta0"], rtol=1e-13, atol=0)
    assert np.allclose(lib["S0"], ref["S0"], rtol=1e-13, atol=0)
    assert abs(lib["Sg0"] - ref["Sg0"]) < 1e-12 * ref["Sg0"]
    assert abs(lib["V0"] - ref["V0"]) < 1e-12 * ref["V0"]


def test_mesh_check_rejections():
    nodes, tris = mesh.icosphere(1)
    cases = {
        "open": (nodes, tris[:-1]),
        "outward": (nodes, tris[:, [0, 2, 1]]),
        "inconsistent": (nodes, np.vstack([tris[:1, [0, 2, 1]], tris[1:]])),
        "unused node": (np.vstack([nodes, [[5.0, 5.0, 5.0]]]), tris),
        "bad id": (nodes, np.where(tris == 3, 999, tris)),
    }
    for name, (n, t) in cases.items():
        with pytest.raises(lbib.LbibError) as ei:
            lbib.lbib_mesh_check(n, t)
        assert ei.value.status in (-3, -1), name
    with pytest.raises(lbib.LbibError):
        lbib.lbib_mesh_check(nodes[:3], tris[:1])


def test_footprint_accounts_for_storage_precision():
    p32 = lbib.fluid_params(256, 128, 128, precision="f32")
    p16 = lbib.fluid_params(256, 128, 128, precision="f16s")
    b32 = lbib.lbib_footprint_bytes(p32, 0, 0)
    b16 = lbib.lbib_footprint_bytes(p16, 0, 0)
    nf = 256 * 126 * 128
    assert b32 >= 2 * 19 * 4 * nf and b16 >= 2 * 19 * 2 * nf
    assert b32 - b16 >= 2 * 19 * 2 * nf
    assert lbib.lbib_footprint_bytes(p32, 1000, 2000) > b32


def test_server_host_logic_without_gpu():
    """The scheduler's argument checks and empty-state behaviour are host
    code: no device call happens before a simulation is admitted."""
    with pytest.raises(lbib.LbibError):
        lbib.lbib_server_create(0, 4, 16)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_server_create(1 << 30, 0, 16)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_server_create(1 << 30, 4, 0)
    srv = lbib.lbib_server_create(1 << 30, 4, 16)
    try:
        assert lbib.lbib_server_stats(srv) == dict(resident=0, resident_bytes=0, advances=0, updates=0)
        assert lbib.lbib_server_advance(srv) == []
        assert lbib.lbib_server_stats(srv)["advances"] == 0
    finally:
        lbib.lbib_server_destroy(srv)


def test_bounded_wait_check_argument_errors_without_gpu():
    """The wait check rejects a bound outside (0, 10] s before any device call."""
    for sec in (0.0, -1.0, 11.0, float("nan")):
        with pytest.raises(lbib.LbibError) as e:
            lbib.lbib_check_bounded_wait(sec)
        assert e.value.status == lbib.LBIB_ERR_ARG


def test_mesh_orientation_check_repair_flip():
    """Sec. 5 mesh analysis: a consistently inward mesh needs no change;
    flipping every triangle is undone by the repair; a random subset of
    turned triangles of a concave (biconcave) mesh is repaired exactly."""
    for nodes, tris in (mesh.icosphere(2), mesh.biconcave(3)):
        t = np.asarray(tris, dtype=np.int32)
        _, n = lbib.lbib_mesh_orient(nodes, t, lbib.MESH_CHECK)
        assert n == 0
        fl, n = lbib.lbib_mesh_orient(nodes, t, lbib.MESH_FLIP)
        assert n == len(t) and np.array_equal(fl[:, [0, 2, 1]], t)
        rep, n = lbib.lbib_mesh_orient(nodes, fl, lbib.MESH_REPAIR)
        assert n == len(t) and np.array_equal(rep, t)
        rng = np.random.default_rng(5)
        sel = rng.random(len(t)) < 0.3
        bad = t.copy()
        bad[sel] = bad[sel][:, [0, 2, 1]]
        _, n = lbib.lbib_mesh_orient(nodes, bad, lbib.MESH_CHECK)
        assert n == int(sel.sum())
        rep, _ = lbib.lbib_mesh_orient(nodes, bad, lbib.MESH_REPAIR)
        assert np.array_equal(rep, t)
        lbib.lbib_mesh_check(nodes, rep)   # accepted as a template


def test_mesh_orientation_rejects_open_mesh():
    nodes, tris = mesh.icosphere(1)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_mesh_orient(nodes, np.asarray(tris[1:], dtype=np.int32), lbib.MESH_REPAIR)


def test_vtk_roundtrip(tmp_path):
    from paper_1312_3426_gb300 import vtk
    nodes, tris = mesh.biconcave(2)
    p = tmp_path / "cell.vtk"
    vtk.write_vtk(p, nodes * 8.0, tris, {"speed": np.arange(len(nodes), dtype=float)})
    X, T = vtk.read_vtk(p)
    assert np.array_equal(X, nodes * 8.0) and np.array_equal(T, tris)


# The largest box: population indices are 32-bit (19 x padded cells < 2^32).
MAX_BOX = (1024, 217, 1024)  # walls in y: 215 fluid rows, 225,443,840 fluid cells


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_largest_box_accepted_one_row_more_refused(prec):
    nx, ny, nz = MAX_BOX
    nf = nx * (ny - 2) * nz
    assert 19 * nf < 2 ** 32 <= 19 * nx * (ny - 1) * nz
    esz = 4 if prec == "f32" else 2
    ok = lbib.lbib_footprint_bytes(lbib.fluid_params(nx, ny, nz, precision=prec), 0, 0)
    assert ok >= 2 * 19 * esz * nf + 3 * 16 * nf
    too_big = lbib.fluid_params(nx, ny + 1, nz, precision=prec)
    assert lbib.lbib_footprint_bytes(too_big, 0, 0) == -1
    with pytest.raises(lbib.LbibError) as e:  # refused before any device call
        lbib.lbib_create(too_big)
    assert e.value.status == lbib.LBIB_ERR_ARG
