"""Bounds of the lattice-index arithmetic of the immersed-boundary coupling
(interpolation corners and the 4x4x4 marking halo of Sec. 2's velocity
interpolation and drag spreading), on the host.

The library's own index functions (csrc/lattice_index.h, compiled for host
and device from the same source) are driven by a small host program with
the node positions of the seeded serving trace (256 channel requests of
32^3 .. 192x96x96 cells with up to 100 red-cell meshes each), the same
positions displaced far outside their boxes, and hand-picked special
values: non-finite and saturated coordinates, +-2^31, values on lattice
planes, large or non-finite low parts.  Every index a node kernel would
touch must be -1 (solid row) or a fluid cell below nx nyf nz, and every
mask word below the word count.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1312_3426_gb300", "csrc")
SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice_index_bounds.cpp")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("lattice_index") / "lattice_index_bounds")
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Werror", "-I", CSRC, SRC, "-o", exe], check=True)
    return exe


def run(driver, box, walls, xyz_hi, xyz_lo=None):
    """xyz_hi, xyz_lo: [n, 3] float32; returns the driver's counters."""
    hi = np.asarray(xyz_hi, np.float32).reshape(-1, 3)
    lo = np.zeros_like(hi) if xyz_lo is None else np.asarray(xyz_lo, np.float32).reshape(-1, 3)
    rec = np.empty((len(hi), 6), np.float32)
    rec[:, 0::2] = hi
    rec[:, 1::2] = lo
    p = subprocess.run([driver, *map(str, box), str(int(walls))], input=rec.tobytes(), capture_output=True,
                       check=True)
    keys = ("nodes", "skipped", "corner_refs", "halo_refs", "bad", "max_index", "max_word", "nf", "nwords")
    return dict(zip(keys, map(int, p.stdout.split())))


def check(r, n):
    assert r["nodes"] == n
    assert r["bad"] == 0, r
    assert r["max_index"] < r["nf"] and r["max_word"] < r["nwords"], r


def split_hi_lo(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def rotation(r):
    cx, sx, cy, sy, cz, sz = np.cos(r[0]), np.sin(r[0]), np.cos(r[1]), np.sin(r[1]), np.cos(r[2]), np.sin(r[2])
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def scene_nodes(sc):
    out = []
    for ob in sc.objects:
        t = sc.templates[ob.tid]
        x = t.nodes * np.asarray(t.stretch)
        out.append(x @ rotation(ob.rotate).T + np.asarray(ob.origin))
    return np.concatenate(out) if out else np.zeros((0, 3))


@pytest.fixture(scope="module")
def trace():
    sys.path.insert(0, ROOT)
    from workloads import scenes
    return scenes.serving_trace(n_requests=256, seed=4, rate_per_s=1.0)


def test_serving_trace_positions_stay_in_bounds(driver, trace):
    rng = np.random.default_rng(11)
    boxes = 0
    for req in trace:
        sc = req.scene
        X = scene_nodes(sc)
        if len(X) == 0:
            continue
        box = (sc.nx, sc.ny, sc.nz)
        # as placed, then carried anywhere in and far outside the box
        far = X + rng.uniform(-3.0, 3.0, (len(X), 3)) * np.array(box)
        huge = X * rng.choice([1e3, 1e7, 1e12, -1e20], size=(len(X), 1))
        for P in (X, far, huge):
            hi, lo = split_hi_lo(P)
            r = run(driver, box, sc.walls, hi, lo)
            check(r, len(P))
            assert r["skipped"] == 0
        boxes += 1
    assert boxes >= 200  # nearly every request carries cells


@pytest.mark.parametrize("walls", [True, False])
@pytest.mark.parametrize("box", [(32, 32, 32), (33, 35, 37), (192, 96, 96), (1, 3, 1), (2, 1, 2)])
def test_special_coordinates_stay_in_bounds(driver, box, walls):
    if walls and box[1] < 3:
        pytest.skip("a walled channel needs at least one fluid row")
    nx, ny, nz = box
    f = np.float32
    specials = np.array([0.0, -0.0, 0.5, -0.5, 1.0, 1.5, ny - 1.5, ny - 1.0, ny - 0.5, ny, ny + 0.5,
                         nx - 0.5, nz - 0.5, 2.0 ** 22 + 0.5, 2.0 ** 24, 2.0 ** 30, 2.0 ** 31, -2.0 ** 31,
                         2.0 ** 31 + 4096, 3.0e9, -3.0e9, 1e30, -1e30, 3.4e38, -3.4e38, 1e-45, -1e-45,
                         np.nextafter(f(0.5), f(1)), np.nextafter(f(0.5), f(0)),
                         np.nextafter(f(ny - 1.5), f(0)), np.inf, -np.inf, np.nan], np.float64)
    lows = np.array([0.0, 0.49, -0.49, 0.999, -0.999, 3.0, -3.0, 1e30, -1e30, np.inf, -np.inf, np.nan])
    rng = np.random.default_rng(12)
    n = 20000
    hi = rng.choice(specials, size=(n, 3)).astype(np.float32)
    lo = rng.choice(lows, size=(n, 3)).astype(np.float32)
    r = run(driver, box, walls, hi, lo)
    check(r, n)
    finite = np.isfinite(hi).all(axis=1)
    assert r["skipped"] == int((~finite).sum())  # non-finite positions touch nothing
    assert r["corner_refs"] > 0 and r["halo_refs"] > 0
    # every combination of one special per axis with no low part
    g = np.array(np.meshgrid(specials, specials, specials, indexing="ij")).reshape(3, -1).T
    r = run(driver, box, walls, g.astype(np.float32))
    check(r, len(g))


def test_corners_of_interior_points_are_the_expected_cells(driver):
    """A node strictly inside a walled channel touches exactly its 8 corner
    cells and a 4x4x4 halo (no solid row within reach)."""
    box = (16, 12, 10)
    X = np.array([[5.7, 5.2, 4.9]], np.float32)
    r = run(driver, box, True, X)
    assert r["corner_refs"] == 8 and r["halo_refs"] == 64 and r["bad"] == 0
    # next to the wall (y in the first fluid cell): the lower corners fall on
    # the solid row and the halo loses its solid rows
    r = run(driver, box, True, np.array([[5.7, 1.2, 4.9]], np.float32))
    assert r["corner_refs"] == 4 and r["halo_refs"] == 32

