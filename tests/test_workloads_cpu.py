"""The seeded input recipes the benchmark and tests use (workloads/): they
are deterministic and have the sizes, spacings and counts the design notes
quote.  Inputs only: none of the method's arithmetic is here."""
import numpy as np

from workloads import mesh, scenes


def _min_image_separation(sc):
    c = np.array([o.origin for o in sc.objects])
    box = np.array([sc.nx, sc.ny, sc.nz], dtype=np.float64)
    best = np.inf
    for i in range(len(c)):
        d = c[i + 1:] - c[i]
        for ax in (0, 2):
            d[:, ax] -= box[ax] * np.round(d[:, ax] / box[ax])
        if len(d):
            best = min(best, float(np.sqrt(np.einsum("ij,ij->i", d, d)).min()))
    return best


def test_channel_rbc_recipe():
    sc = scenes.channel_rbc()
    assert (sc.nx, sc.ny, sc.nz) == (256, 128, 128) and sc.walls
    assert len(sc.objects) == 200 and sc.n_nodes == 128_400 and sc.n_fluid_cells == 4_128_768
    r = sc.templates[0].stretch[0]
    assert r == 8.0
    assert _min_image_separation(sc) >= 2 * r + 2
    y = np.array([o.origin[1] for o in sc.objects])
    assert y.min() >= 1 + r + 2 and y.max() <= sc.ny - 1 - r - 2
    again = scenes.channel_rbc()
    assert [o.origin for o in again.objects] == [o.origin for o in sc.objects]
    assert [o.rotate for o in again.objects] == [o.rotate for o in sc.objects]


def test_batch_mix_recipe():
    scs = scenes.batch_mix(64)
    assert len(scs) == 64
    assert sum(len(s.objects) for s in scs) == 704
    assert sum(s.n_nodes for s in scs) == 618_048
    assert sum(s.n_fluid_cells for s in scs) == 7_882_849
    levels = set()
    for s in scs:
        assert 32 <= s.nx <= 128 and 32 <= s.ny <= 64 and 32 <= s.nz <= 64
        assert len(s.objects) <= 40
        t = s.templates[0]
        levels.add(len(t.nodes))
        x = t.nodes * np.array(t.stretch)
        e = np.concatenate([np.linalg.norm(x[t.tris[:, a]] - x[t.tris[:, b]], axis=1)
                            for a, b in ((0, 1), (1, 2), (2, 0))])
        assert e.mean() >= 0.49          # the stability floor of the membrane update
        if len(s.objects) > 1:
            assert _min_image_separation(s) >= 2 * t.stretch[0] + 2
    assert levels == {162, 642, 2562}    # levels 2, 3 and 4 all occur
    again = scenes.batch_mix(8)  # the same seeded sequence: a prefix of the 64
    assert [(s.nx, s.ny, s.nz, [o.origin for o in s.objects]) for s in again] == \
        [(s.nx, s.ny, s.nz, [o.origin for o in s.objects]) for s in scs[:8]]


def test_serving_trace_recipe():
    reqs = scenes.serving_trace(256, seed=4, rate_per_s=10.0)
    assert len(reqs) == 256
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.1) < 0.02       # Poisson gaps with mean 1/rate
    for r in reqs:
        s = r.scene
        assert 32 <= s.nx <= 192 and 32 <= s.ny <= 96 and 32 <= s.nz <= 96
        assert 1000 <= r.steps <= 20000 and 1 <= len(s.objects) <= 100
    again = scenes.serving_trace(32, seed=4, rate_per_s=10.0)
    key = lambda r: (r.arrival_s, r.steps, r.scene.nx)  # noqa: E731
    assert [key(r) for r in again] == [key(r) for r in reqs[:32]]


def test_octasphere_counts_closed_and_inward():
    """4 * 4^L + 2 nodes and 8 * 4^L triangles on the unit sphere; every edge
    shared by exactly two triangles (V - E + F = 2); inward orientation
    (negative signed volume sum A . (B x C) for the inward reading); the
    enclosed volume rises from the octahedron's 4/3 towards the sphere's."""
    prev = 0.0
    for level in range(4):
        nodes, tris = mesh.octasphere(level)
        assert len(nodes) == 4 * 4 ** level + 2 and len(tris) == 8 * 4 ** level
        assert np.allclose(np.linalg.norm(nodes, axis=1), 1.0)
        edges = {}
        for a, b, c in tris:
            for i, j in ((a, b), (b, c), (c, a)):
                edges[(min(i, j), max(i, j))] = edges.get((min(i, j), max(i, j)), 0) + 1
        assert set(edges.values()) == {2}
        assert len(nodes) - len(edges) + len(tris) == 2
        a, b, c = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
        v6 = float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum())
        assert v6 < 0.0
        vol = -v6 / 6.0  # the regular octahedron of unit circumradius has volume 4/3
        assert (abs(vol - 4.0 / 3.0) < 1e-12) if level == 0 else (prev < vol < 4.0 / 3.0 * np.pi)
        prev = vol
    assert vol > 0.97 * 4.0 / 3.0 * np.pi
