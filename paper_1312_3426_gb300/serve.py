"""Request loop over the continuous-batching scheduler.

``run_trace`` replays a trace of channel-simulation requests (arrival time,
scene, step count) in real time on one GPU, in one of two modes:

``batched``  continuous batching: requests that have arrived are admitted in
             arrival order as soon as a resident slot and enough of the
             device-memory budget are free (``lbib_server_admit``); every
             resident simulation advances together by one batched call per
             chunk of steps (``lbib_server_advance`` ->
             ``lbib_batch_step``), and a simulation is retired, read out and
             freed the moment its step count is reached.
``fifo``     the plain loop: one request at a time, in arrival order, each
             run to completion alone (``lbib_step``).

Latency of a request = completion time - arrival time (queueing included).
Aggregate throughput = lattice updates of all requests / (last completion -
first arrival).  All device work goes through the C ABI.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lbib


@dataclass
class Outcome:
    rid: int
    arrival: float
    admitted: float = 0.0
    done: float = 0.0
    cells: int = 0
    steps: int = 0
    failed: str = ""   # status message of a simulation that failed

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class TraceResult:
    mode: str
    outcomes: list = field(default_factory=list)
    wall_s: float = 0.0
    updates: int = 0
    max_resident: int = 0
    max_resident_bytes: int = 0

    def percentile(self, q):
        return float(np.percentile([o.latency for o in self.outcomes], q)) if self.outcomes else 0.0

    @property
    def mlups(self):
        return self.updates / self.wall_s / 1e6 if self.wall_s > 0 else 0.0

    def summary(self):
        return {"mode": self.mode, "requests": len(self.outcomes),
                "failed": sum(1 for o in self.outcomes if o.failed), "p50_s": round(self.percentile(50), 4),
                "p99_s": round(self.percentile(99), 4), "mean_s": round(float(np.mean(
                    [o.latency for o in self.outcomes])) if self.outcomes else 0.0, 4),
                "wall_s": round(self.wall_s, 3), "mlups": round(self.mlups, 1),
                "max_resident": self.max_resident, "max_resident_gb": round(self.max_resident_bytes / 1e9, 3)}


def _footprint(req, precision, pop_scale_log2):
    sc = req.scene
    p = lbib.fluid_params(sc.nx, sc.ny, sc.nz, sc.walls, sc.tau, sc.rho0, sc.body_force, sc.friction,
                          precision, pop_scale_log2)
    tris = sum(len(sc.templates[o.tid].tris) for o in sc.objects)
    return lbib.lbib_footprint_bytes(p, sc.n_nodes, tris)


def run_trace(requests, mode="batched", precision="f16s", pop_scale_log2=12, budget_bytes=150e9,
              max_resident=64, chunk_steps=256, stream=None, on_done=None, time_scale=1.0):
    """Replays `requests` (objects with rid, arrival_s, scene, steps).
    on_done(rid, sim) is called with each finished simulation before it is
    freed.  time_scale multiplies the arrival times (0: all at once)."""
    reqs = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
    res = TraceResult(mode)
    out = {r.rid: Outcome(r.rid, r.arrival_s * time_scale, cells=r.scene.n_fluid_cells, steps=r.steps) for r in reqs}
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0  # noqa: E731

    if mode == "fifo":
        for r in reqs:
            o = out[r.rid]
            wait = o.arrival - now()
            if wait > 0:
                time.sleep(wait)
            o.admitted = now()
            sim = lbib.Sim.from_scene(r.scene, precision=precision, pop_scale_log2=pop_scale_log2, stream=stream)
            sim.step(r.steps)
            try:
                sim.sync()
            except lbib.LbibError as err:
                o.failed = str(err)
            o.done = now()
            res.max_resident = 1
            res.max_resident_bytes = max(res.max_resident_bytes, int(sim.info()[5]))
            if on_done and not o.failed:
                on_done(r.rid, sim)
            sim.close()
            if not o.failed:
                res.updates += o.cells * o.steps
            res.outcomes.append(o)
    elif mode == "batched":
        srv = lbib.lbib_server_create(int(budget_bytes), max_resident, chunk_steps)
        try:
            pending = []      # arrived, not admitted (arrival order)
            resident = {}     # rid -> Sim
            nxt = 0
            while nxt < len(reqs) or pending or resident:
                t = now()
                while nxt < len(reqs) and out[reqs[nxt].rid].arrival <= t:
                    pending.append(reqs[nxt])
                    nxt += 1
                # admit in arrival order while the head fits
                while pending:
                    r = pending[0]
                    st = lbib.lbib_server_stats(srv)
                    if st["resident"] >= max_resident or st["resident_bytes"] + _footprint(
                            r, precision, pop_scale_log2) > budget_bytes:
                        break
                    sim = lbib.Sim.from_scene(r.scene, precision=precision, pop_scale_log2=pop_scale_log2,
                                              stream=stream)
                    if not lbib.lbib_server_admit(srv, sim.h, r.steps, r.rid):
                        sim.close()
                        break
                    resident[r.rid] = sim
                    out[r.rid].admitted = now()
                    pending.pop(0)
                if not resident:
                    if nxt < len(reqs):
                        time.sleep(max(0.0, out[reqs[nxt].rid].arrival - now()))
                    continue
                st = lbib.lbib_server_stats(srv)
                res.max_resident = max(res.max_resident, st["resident"])
                res.max_resident_bytes = max(res.max_resident_bytes, st["resident_bytes"])
                for rid in lbib.lbib_server_advance(srv):
                    sim = resident.pop(rid)
                    o = out[rid]
                    try:
                        sim.sync()
                    except lbib.LbibError as err:
                        o.failed = str(err)
                    if on_done and not o.failed:
                        on_done(rid, sim)
                    o.done = now()
                    sim.close()
                    if not o.failed:
                        res.updates += o.cells * o.steps
                    res.outcomes.append(o)
        finally:
            lbib.lbib_server_destroy(srv)
    else:
        raise ValueError(f"unknown mode {mode!r}")
    first = min(o.arrival for o in out.values()) if out else 0.0
    res.wall_s = max((o.done for o in res.outcomes), default=0.0) - first
    return res
