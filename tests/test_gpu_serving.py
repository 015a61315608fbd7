"""Continuous batching: the scheduler (lbib_server_*) and the request loop
(serve.run_trace) on small synthetic channel requests.

A request's result does not depend on what else is resident: the batched
step runs the same per-item device code as lbib_step, so a simulation
served in the mix matches the same simulation stepped alone up to the
order of the FP32 atomics (FP32 storage: fluid relative L2 <= 1e-5, nodes
<= 1e-6 lu; FP16 storage: the stochastic-rounding bits are keyed by cell
and step and are the same in both runs, but an atomic-order difference can
flip a rounding decision, so the FP16 bar, 1e-3 relative L2, applies).
"""
from dataclasses import dataclass

import numpy as np
import pytest

from paper_1312_3426_gb300 import lbib, serve
from workloads import mesh, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1312_3426_gb300 import build
    build.build()
    lbib.load()


@dataclass
class Req:
    rid: int
    arrival_s: float
    scene: object
    steps: int


def small_trace(n=7, seed=11):
    rng = np.random.default_rng(seed)
    nodes, tris = mesh.biconcave(2)
    out = []
    for i in range(n):
        nx, ny, nz = int(rng.integers(20, 41)), int(rng.integers(16, 25)), int(rng.integers(16, 25))
        sc = scenes.Scene(f"r{i}", nx, ny, nz, body_force=(2e-5, 0.0, 0.0))
        sc.templates.append(scenes.Template(nodes, tris, (3.0, 3.0, 3.0), **scenes.PAPER_MODULI))
        for c in scenes.place_spheres(rng, nx, ny, nz, 3.0, int(rng.integers(0, 3)), max_tries=500):
            sc.objects.append(scenes.Obj(0, tuple(float(v) for v in c), scenes.random_rotation(rng)))
        out.append(Req(i, 0.0, sc, int(rng.integers(30, 90))))
    return out


def rel_l2(a, b, ny):
    a = a[:, :, 1:ny - 1, :].astype(np.float64)
    b = b[:, :, 1:ny - 1, :].astype(np.float64)
    return float(np.linalg.norm(a - b) / max(1e-30, np.linalg.norm(b)))


@pytest.mark.parametrize("prec,scale,tol_u,tol_x", [("f32", 0, 1e-5, 1e-6), ("f16s", 12, 1e-3, 1e-4)])
def test_served_result_equals_alone(prec, scale, tol_u, tol_x):
    reqs = small_trace()
    assert any(r.scene.objects for r in reqs) and any(not r.scene.objects for r in reqs)
    got = {}

    def keep(rid, sim):
        got[rid] = (sim.velocity(), sim.read_nodes(-1)[0] if sim.obj_tid else None)

    # three slots and short chunks: requests join and leave while others run
    r = serve.run_trace(reqs, "batched", precision=prec, pop_scale_log2=scale, max_resident=3, chunk_steps=8,
                        on_done=keep, time_scale=0.0)
    assert len(r.outcomes) == len(reqs) and r.max_resident == 3
    for q in reqs:
        alone = lbib.Sim.from_scene(q.scene, precision=prec, pop_scale_log2=scale)
        alone.step(q.steps)
        u, x = got[q.rid]
        assert rel_l2(u, alone.velocity(), q.scene.ny) <= tol_u, q.rid
        if x is not None:
            assert np.abs(x - alone.read_nodes(-1)[0]).max() <= tol_x, q.rid
        alone.close()


def test_budget_caps_resident_memory():
    reqs = small_trace(5, seed=12)
    need = max(serve._footprint(q, "f16s", 12) for q in reqs)
    budget = int(1.5 * need)
    r = serve.run_trace(reqs, "batched", budget_bytes=budget, max_resident=8, chunk_steps=16, time_scale=0.0)
    assert len(r.outcomes) == len(reqs)
    assert r.max_resident_bytes <= budget
    # admission is in arrival order: completion order follows it when one fits at a time
    assert r.max_resident >= 1


def test_fifo_and_batched_same_work():
    reqs = small_trace(6, seed=13)
    a = serve.run_trace(reqs, "fifo", time_scale=0.0)
    b = serve.run_trace(reqs, "batched", time_scale=0.0)
    assert a.updates == b.updates == sum(q.scene.n_fluid_cells * q.steps for q in reqs)
    assert sorted(o.rid for o in a.outcomes) == sorted(o.rid for o in b.outcomes)


def test_server_admission_errors():
    srv = lbib.lbib_server_create(1 << 40, 2, 4)
    try:
        reqs = small_trace(3, seed=14)
        sims = [lbib.Sim.from_scene(q.scene) for q in reqs]
        assert lbib.lbib_server_admit(srv, sims[0].h, 5, 0)
        with pytest.raises(lbib.LbibError):
            lbib.lbib_server_admit(srv, sims[0].h, 5, 0)   # already resident
        assert lbib.lbib_server_admit(srv, sims[1].h, 9, 1)
        assert not lbib.lbib_server_admit(srv, sims[2].h, 5, 2)  # no slot
        assert lbib.lbib_server_advance(srv) == []        # 4 steps each
        assert lbib.lbib_server_advance(srv) == [0]       # 1 step: request 0 done
        assert lbib.lbib_server_admit(srv, sims[2].h, 5, 2)
        done = []
        while lbib.lbib_server_stats(srv)["resident"]:
            done += lbib.lbib_server_advance(srv)
        assert sorted(done) == [1, 2]
        assert [int(s.info()[4]) for s in sims] == [5, 9, 5]
    finally:
        lbib.lbib_server_destroy(srv)


def test_batch_plan_follows_new_simulations():
    """A simulation created where a destroyed one lived (same address, same
    object count) must get its own work list."""
    for i in range(4):
        sc = scenes.Scene(f"b{i}", 20 + 6 * i, 18, 14 + 2 * i, body_force=(2e-5, 0.0, 0.0))
        g = lbib.Sim.from_scene(sc)
        lbib.lbib_batch_step([g.h], 40)
        a = lbib.Sim.from_scene(sc)
        a.step(40)
        assert rel_l2(g.velocity(), a.velocity(), sc.ny) <= 1e-6
        g.close()
        a.close()


def test_failed_simulation_retires_alone():
    reqs = small_trace(4, seed=15)
    # an unstable request: a body force far beyond the lattice's range
    reqs[1].scene.body_force = (5e-2, 0.0, 0.0)
    reqs[1].steps = 400
    r = serve.run_trace(reqs, "batched", precision="f32", pop_scale_log2=0, max_resident=4, chunk_steps=16,
                        time_scale=0.0)
    failed = {o.rid for o in r.outcomes if o.failed}
    assert failed == {1}
    assert len(r.outcomes) == 4
