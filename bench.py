#!/usr/bin/env python3
"""Throughput of the fused LB-IB step on one GB300 (or N replicas).

A step is one pass of the whole hot path over the workload: interpolation,
drag, spreading and node update (one thread per node), then the fused D3Q19
pull-stream + BGK/Guo collide with bounce-back walls (one kernel); the
per-object area and volume sums and the five membrane forces of the next
step (one thread-block cluster per object) run on a second stream beside
the fluid kernel.  The default workload is the
256x128x128 channel with 200 Evans-Fung red blood cells (level-3 meshes,
128,400 nodes), FP32 populations; the populations (628 MB) exceed the L2
cache, so no flush is needed between steps.

Printed JSON line (rank 0):
  value        MLUPS = fluid lattice updates per second / 1e6, all ranks
  roofline     fluid kernel: 152 B (FP32) or 76 B (FP16/BF16) per fluid cell
               per launch / its mean CUDA-event duration, against the
               measured copy bandwidth
  e2e          the same metric through the public C ABI with a host loop:
               every step uploads the per-object external forces from pinned
               host memory, steps, and reads every object's analysis back
               (step k's analysis read while step k+1 runs; the loop that
               waits every step is reported beside it)
  cpu_baseline the FP64 oracle on the host cores, a bounded number of full
               steps of the same workload
  serving      a seeded Poisson trace of 256 channel requests (FP16-shifted
               storage, 150 GB budget) served by continuous batching
               (lbib_server_*) and by the plain one-at-a-time loop: p50/p99
               completion latency and aggregate MLUPS of both
``--impl reference`` times that oracle alone on the same workload;
``--workload batch64`` measures 64 independent channels advanced together.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LB+IB MLUPS & %HBM roofline, FP32 vs FP16-store; serving p50/p99 vs plain"
BYTES_PER_CELL = {"f32": 152, "f16s": 76, "bf16s": 76}
FLUID_KERNELS = ("k_fluid", "k_fluid_pair", "k_fluid_pair_tma")
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["rbc256", "rbc512", "sphere40", "batch64"], default="rbc256")
    ap.add_argument("--precision", choices=["f32", "f16s", "bf16s"], default="f32")
    ap.add_argument("--scale-log2", type=int, default=12, help="storage scale 2^s for f16s/bf16s")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ib-cluster", type=int, default=0, help="thread blocks per object (0: library default)")
    ap.add_argument("--overlap", type=int, default=-1, choices=(-1, 0, 1),
                    help="membrane forces overlapped with the fluid step (-1: library default)")
    ap.add_argument("--membrane-clusters", type=int, default=-1,
                    help="clusters of the membrane kernel (0: one per object, -1: library default)")
    ap.add_argument("--membrane-threads", type=int, default=0,
                    help="block size of the membrane kernel (0: library default)")
    ap.add_argument("--node-threads", type=int, default=0, help="nodes per block of the node kernel (0: default)")
    ap.add_argument("--membrane-group", type=int, default=0, help="objects per membrane block (0: library default)")
    ap.add_argument("--early-launch", type=int, default=-1, choices=(-1, 0, 1),
                    help="programmatic dependent launch of the node and fluid kernels (-1: library default)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's launch shapes (and the flags above) instead of autotuning them")
    ap.add_argument("--fluid-kernel", type=int, default=-1, choices=(-1, 0, 1, 2, 3),
                    help="16-bit fluid kernel (-1: library default; see LBIB_TUNE_FLUID_KERNEL)")
    ap.add_argument("--launch", choices=["separate", "batched"], default="separate",
                    help="lbib_step, or lbib_batch_step (work lists + captured graphs) on the one simulation")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving comparison")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP32 / FP16-shifted / BF16-shifted records (both RBC channels, Poiseuille error)")
    ap.add_argument("--no-poiseuille", action="store_true",
                    help="skip the Poiseuille errors (20,000 steps of the object-free 512x256x256 channel per storage)")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-mlups-estimate", type=float, default=22000.0,
                    help="batched FP16 throughput used to set the arrival rate (offered load 0.8)")
    return ap.parse_args()


def make_scene(name):
    from workloads import scenes
    if name == "rbc256":
        return scenes.channel_rbc()
    if name == "rbc512":
        return scenes.channel_rbc_large()
    return scenes.channel_sphere()


def workload_desc(sc):
    return (f"{sc.name}: {len(sc.objects)} objects, {sc.n_nodes} nodes, "
            f"{sc.n_fluid_cells} fluid cells, tau={sc.tau}, body force {sc.body_force[0]:g}")


def max_over_ranks(x, device=None):
    """The largest of x over all ranks of the default process group (x
    itself without one); device: where the reduction tensor lives (the
    rank's GPU for NCCL, None for CPU / gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(units_per_rank, steps, ms_max, world):
    """Replicas: every rank advances its own copy of the workload, so the job
    processes world x units per step in the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3) / 1e6


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    """Hash of the fluid kernel sources without their comments and blank
    lines (a comment edit does not change what was profiled)."""
    h = hashlib.sha256()
    for rel in ("paper_1312_3426_gb300/csrc/fluid_core.cuh", "paper_1312_3426_gb300/csrc/fluid.cu"):
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(workload, precision, cells):
    """DRAM bytes per launch of the fluid kernel from the committed ncu
    summary (lines ``traffic: workload=.. precision=.. source_hash=..
    dram_bytes_per_cell=..``), when it was taken on the current kernel
    source; else None."""
    path = os.path.join(ROOT, "profiles", "k_fluid_dram_traffic.md")
    try:
        with open(path) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if not ln.startswith("traffic:"):
            continue
        kv = dict(tok.split("=", 1) for tok in ln.split()[1:] if "=" in tok)
        if (kv.get("workload") == workload and kv.get("precision") == precision
                and kv.get("source_hash") == kernel_source_hash()):
            return round(float(kv["dram_bytes_per_cell"]) * cells)
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            self.fh = tempfile.NamedTemporaryFile("w", prefix="lbib_clocks_", suffix=".csv", delete=False)
            self.path = self.fh.name
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
            if self.path:
                self.fh.close()
                try:
                    os.unlink(self.path)
                except OSError:
                    pass

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as f:
            lines = f.readlines()
        try:
            os.unlink(self.path)
        except OSError:
            pass
        rows = []
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            if self.uuid and self.uuid not in p[0] and not p[0].endswith(self.uuid):
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(sc, target_s):
    import oracle
    o = oracle.Oracle.from_scene(sc)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    k = max(1, int(target_s / max(t1, 1e-3)) - 1)
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    return {"value": round(sc.n_fluid_cells * k / dt / 1e6, 3), "unit": "MLUPS", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{k} full FP64 steps of {sc.name} after 1 untimed step ({dt:.1f} s)",
            "nodes_per_s": round(sc.n_nodes * k / dt, 1)}


def e2e_record(nf, steps, dt_s, dt_sync_s, world, nobj):
    """The `e2e` object: MLUPS of the host loop that reads step k's analysis
    after enqueueing step k+1, the bytes it moves per step (forces up: 3 FP32
    per object; analysis down: 14 FP64 per object and the status word), and
    the MLUPS of the loop that waits for every step."""
    return {"value": round(whole_job_mlups(nf, steps, dt_s * 1e3, world), 2), "unit": "MLUPS",
            "h2d_bytes_per_step": 12 * nobj, "d2h_bytes_per_step": 14 * 8 * nobj + 4,
            "loop": "per step: forces up from pinned memory, step, analysis + status enqueued into a pinned slot; "
                    "step k's analysis read after step k+1 is enqueued",
            "synchronous_value": round(whole_job_mlups(nf, steps, dt_sync_s * 1e3, world), 2)}


def reference_run(sc, warmup, steps, budget_s=120.0):
    """The FP64 oracle as it stands on the host cores: `warmup` untimed full
    steps (at most 2), then min(steps, as many as fit in budget_s) timed
    full steps of the same workload."""
    import oracle
    o = oracle.Oracle.from_scene(sc)
    t0 = time.perf_counter()
    nw = max(1, min(int(warmup), 2))
    o.step(nw)
    t1 = (time.perf_counter() - t0) / nw
    k = max(1, min(int(steps), int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    return {"value": round(sc.n_fluid_cells * k / dt / 1e6, 3), "unit": "MLUPS", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{k} of the {steps} requested full FP64 steps of {sc.name} after {nw} untimed "
                      f"({dt:.1f} s)", "ms_per_step": dt / k * 1e3}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc = make_scene(args.workload)
    base = reference_run(sc, args.warmup, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(base["ms_per_step"], 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded channel, Evans-Fung RBC meshes)",
            "config": {"workload": workload_desc(sc), "precision_storage": "f64", "parallelism": "host threads"},
            "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": base["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def apply_knobs(args, lbib, sim):
    """The launch-shape knobs given on the command line."""
    if args.ib_cluster:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_IB_CLUSTER, args.ib_cluster)
    if args.overlap >= 0:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_OVERLAP, args.overlap)
    if args.membrane_clusters >= 0:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_MEMBRANE_CLUSTERS, args.membrane_clusters)
    if args.fluid_kernel >= 0:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_FLUID_KERNEL, args.fluid_kernel)
    if args.membrane_threads:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_MEMBRANE_THREADS, args.membrane_threads)
    if args.node_threads:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_NODE_THREADS, args.node_threads)
    if args.membrane_group:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_MEMBRANE_GROUP, args.membrane_group)
    if args.early_launch >= 0:
        lbib.lbib_set_tuning(sim.h, lbib.LBIB_TUNE_EARLY_LAUNCH, args.early_launch)


def explicit_knobs(args):
    return bool(args.ib_cluster or args.overlap >= 0 or args.membrane_clusters >= 0 or args.fluid_kernel >= 0
                or args.membrane_threads or args.node_threads or args.membrane_group or args.early_launch >= 0)


def batch_workload(args, lbib, torch, dev, stream):
    """64 independent channels (random boxes 32^3..128x64x64, 0-40 cells of
    level 2/3/4, FP32) advanced together by lbib_batch_step; knobs from the
    autotuner, or from the command line (then on every simulation; the batch
    takes the first one's).  Returns the fields of the JSON line."""
    from paper_1312_3426_gb300 import tune
    from workloads import scenes
    scs = scenes.batch_mix(64)
    sims = [lbib.Sim.from_scene(sc, precision=args.precision, pop_scale_log2=args.scale_log2,
                                stream=stream.cuda_stream) for sc in scs]
    for s in sims:
        apply_knobs(args, lbib, s)
    tuning = None
    if not args.no_autotune and not explicit_knobs(args):
        choice, timing = tune.autotune(sims, steps=32, batched=True)
        tuning = dict(choice, candidates_s={k: round(v, 5) for k, v in timing.items()})
    h = [s.h for s in sims]
    lbib.lbib_batch_step(h, max(3, args.warmup))
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lbib.lbib_batch_step(h, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    cells = sum(sc.n_fluid_cells for sc in scs)
    nodes = sum(sc.n_nodes for sc in scs)
    for s in sims:
        s.close()
    return scs, cells, nodes, ms, clocks, tuning


def measure(args, lbib, torch, sc, precision, stream, dev, local, world, barrier, e2e=True, launch="separate",
            clocks=False):
    """Times args.steps steps of scene `sc` with `precision` storage after
    args.warmup untimed ones (CUDA events on the simulation's stream,
    barrier + synchronize on both sides, max over ranks), with per-kernel
    events on every n-th step (n = steps / 8, at most 16, so the fluid
    kernel's mean rests on at least 8 launches); then, with `e2e`, the host
    loop of e2e_record.  Returns the numbers of the JSON line."""
    nf = sc.n_fluid_cells
    tuning = None
    if not args.no_autotune and not explicit_knobs(args):
        # the project's autotuner picks the launch shapes on a copy of the
        # workload (it advances what it times), then the measured simulation
        # starts from the initial state with them
        from paper_1312_3426_gb300 import tune
        probe = lbib.Sim.from_scene(sc, precision=precision, pop_scale_log2=args.scale_log2,
                                    stream=stream.cuda_stream)
        choice, timing = tune.autotune([probe], steps=128, batched=launch == "batched")
        probe.close()
        tuning = dict(choice, candidates_s={k: round(v, 5) for k, v in timing.items()})
    sim = lbib.Sim.from_scene(sc, precision=precision, pop_scale_log2=args.scale_log2, stream=stream.cuda_stream)
    apply_knobs(args, lbib, sim)
    if tuning is not None:
        from paper_1312_3426_gb300 import tune
        tune.apply([sim], tuning)
    kernel = FLUID_KERNELS[int(sim.info()[7])]
    sim.step(max(3, args.warmup))
    sim.sync()
    sampler = None
    if clocks:
        try:
            uuid = str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            uuid = None
        sampler = ClockSampler(uuid)
    barrier()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    persistent = launch == "batched"
    if not persistent:
        lbib.lbib_profile_enable(sim.h, profile_every(args.steps))
    e0.record(stream)
    if persistent:
        lbib.lbib_batch_step([sim.h], args.steps)
    else:
        sim.step(args.steps)
    e1.record(stream)
    barrier()
    clk = sampler.stop() if sampler else None
    prof = lbib.lbib_profile_read(sim.h) if not persistent else None
    lbib.lbib_profile_enable(sim.h, False)
    sim.sync()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    if prof is not None:
        fluid_ms = prof["fluid_ms"] / max(1, prof["fluid_launches"])
        nodes_ms = prof["nodes_ms"] / max(1, prof["nodes_launches"])
        membrane_ms = prof["membrane_ms"] / max(1, prof["membrane_launches"])
        launches = int(prof["fluid_launches"])
    else:  # one fused launch per step: the whole step is the kernel
        fluid_ms, nodes_ms, membrane_ms, launches = ms / args.steps, 0.0, 0.0, args.steps
    rec = None
    if e2e:
        nobj = len(sc.objects)
        fh = torch.zeros((max(nobj, 1), 3), dtype=torch.float64, pin_memory=True).numpy()
        out = torch.zeros((max(nobj, 1), 14), dtype=torch.float64, pin_memory=True).numpy()
        k_e2e = args.steps
        # (1) pipelined host loop: every step uploads its forces, steps and
        # enqueues its analysis; the host reads step k's analysis (two
        # page-locked slots) after enqueueing step k + 1, so the device does
        # not wait for the host between steps
        barrier()
        t0 = time.perf_counter()
        for k in range(k_e2e):
            lbib.lbib_objects_set_force(sim.h, fh[:nobj]) if nobj else None
            sim.step(1)
            lbib.lbib_objects_analyze_async(sim.h, k & 1)
            if k > 0:
                lbib.lbib_objects_analyze_wait(sim.h, (k - 1) & 1, nobj, out)
        lbib.lbib_objects_analyze_wait(sim.h, (k_e2e - 1) & 1, nobj, out)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, dev)
        # (2) the same loop waiting for every step's analysis before the next
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            if nobj:
                lbib.lbib_objects_set_force(sim.h, fh[:nobj])
            sim.step(1)
            if nobj:
                lbib.lbib_objects_analyze(sim.h, nobj, out[:nobj])
            else:
                sim.sync()
        barrier()
        dt_sync = max_over_ranks(time.perf_counter() - t0, dev)
        rec = e2e_record(nf, k_e2e, dt, dt_sync, world, nobj)
    sim.close()
    return {"ms": ms, "value": whole_job_mlups(nf, args.steps, ms, world), "fluid_ms": fluid_ms,
            "nodes_ms": nodes_ms, "membrane_ms": membrane_ms, "fluid_launches": launches, "kernel": kernel,
            "clocks": clk, "e2e": rec, "tuning": tuning}


def profile_every(steps):
    """Per-kernel events on every n-th step: n = steps / 8 (at most 16), so
    that at least 8 fluid launches are timed even in a short run."""
    return max(1, min(16, steps // 8))


GOLDEN_PROFILE = os.path.join(ROOT, "tests", "golden", "channel_512x256x256_profile.txt")


def poiseuille_errors(args, lbib, precisions):
    """Relative L2 of each storage precision's velocity field against the
    FP64 oracle's profile, on the object-free 512x256x256 channel (walls in
    y, tau = 1, body force 1e-5) after 20,000 steps from rest, and the drift
    of its total mass.  The reference profile u_x(y) is the committed file
    tests/golden/channel_512x256x256_profile.txt (written by the oracle;
    the flow is invariant along x and z, and u_y = u_z = 0)."""
    nx, ny, nz, steps = 512, 256, 256, 20000
    prof = np.loadtxt(GOLDEN_PROFILE)
    out = {"steps": steps, "reference": "tests/golden/channel_512x256x256_profile.txt (FP64 oracle)"}
    for prec in precisions:
        g = lbib.Sim(nx, ny, nz, walls=True, tau=1.0, rho0=1.0, body_force=(1e-5, 0.0, 0.0), friction=0.05,
                     precision=prec, pop_scale_log2=0 if prec == "f32" else args.scale_log2)
        g.fluid_init()
        m0 = g.mass()
        g.step(steps)
        m1 = g.mass()
        u = g.velocity()
        g.close()
        num = float(np.sum((u[0][:, 1:ny - 1, :].astype(np.float64) - prof[None, 1:ny - 1, None]) ** 2))
        num += float(np.sum(u[1][:, 1:ny - 1, :].astype(np.float64) ** 2) + np.sum(u[2][:, 1:ny - 1, :].astype(np.float64) ** 2))
        den = float(np.sum(prof[1:ny - 1] ** 2)) * nx * nz
        out[prec] = {"rel_l2": float(f"{(num / den) ** 0.5:.4g}"), "mass_drift": float(f"{abs(m1 - m0) / m0:.3g}")}
    return out


def precision_records(args, lbib, torch, stream, dev, local, world, barrier, peak, main):
    """The FP32 / FP16-shifted / BF16-shifted comparison: MLUPS, the fluid
    kernel's roofline and the end-to-end loop for each storage on the
    256x128x128 channel with 200 cells (the main line's workload) and on the
    512x256x256 channel with 2000 cells, and the Poiseuille error of each
    against the FP64 oracle (object-free 512x256x256 channel)."""
    out = {}
    for wl in ("rbc256", "rbc512"):
        sc = make_scene(wl)
        rows = {}
        for prec in ("f32", "f16s", "bf16s"):
            if wl == args.workload and prec == args.precision and args.launch == "separate":
                m = main
            else:
                m = measure(args, lbib, torch, sc, prec, stream, dev, local, world, barrier,
                            e2e=(wl == "rbc256" and not args.no_e2e))
            bpc = BYTES_PER_CELL[prec]
            ach = bpc * sc.n_fluid_cells / (m["fluid_ms"] / 1e3) / 1e9
            rows[prec] = {"value": round(m["value"], 2), "unit": "MLUPS", "ms_per_step": round(m["ms"] / args.steps, 5),
                          "roofline": {"kernel": f"{m['kernel']}<{prec}>", "bytes_per_cell": bpc,
                                       "mean_launch_ms": round(m["fluid_ms"], 5), "launches_timed": m["fluid_launches"],
                                       "achieved": round(ach, 1), "frac": round(ach / peak, 4)},
                          "step_hbm_frac": round((bpc * sc.n_fluid_cells + 400 * sc.n_nodes) / (m["ms"] / args.steps / 1e3)
                                                 / 1e9 / peak, 4),
                          "e2e": m["e2e"]["value"] if m["e2e"] else None,
                          "tuning": {k: v for k, v in (m["tuning"] or {}).items() if k != "candidates_s"} or None}
        out[workload_desc(sc)] = rows
    if not args.no_poiseuille:
        out["poiseuille_512x256x256"] = poiseuille_errors(args, lbib, ("f32", "f16s", "bf16s"))
    return out


def serving_comparison(args, stream):
    """The request trace served by continuous batching and by the plain
    one-at-a-time loop (same trace, FP16-shifted storage, 150 GB budget)."""
    from paper_1312_3426_gb300 import serve
    from workloads import scenes
    probe = scenes.serving_trace(n_requests=args.serve_requests, seed=4, rate_per_s=1.0)
    mean_work = sum(r.scene.n_fluid_cells * r.steps for r in probe) / len(probe)
    rate = 0.8 * args.serve_mlups_estimate * 1e6 / mean_work
    reqs = scenes.serving_trace(n_requests=args.serve_requests, seed=4, rate_per_s=rate)
    kw = dict(precision="f16s", pop_scale_log2=12, budget_bytes=150e9, stream=stream)
    b = serve.run_trace(reqs, "batched", max_resident=256, chunk_steps=256, **kw)
    f = serve.run_trace(reqs, "fifo", **kw)
    return {"trace": f"{len(reqs)} Poisson arrivals at {rate:.2f}/s (offered load 0.8 of "
                     f"{args.serve_mlups_estimate:.0f} MLUPS), boxes 32^3..192x96x96, 1-100 level-3 RBCs, "
                     f"1k-20k steps, FP16-shifted, 150 GB budget, seed 4",
            "batched": b.summary(), "fifo": f.summary(),
            "p50_speedup": round(f.percentile(50) / max(1e-9, b.percentile(50)), 2),
            "p99_speedup": round(f.percentile(99) / max(1e-9, b.percentile(99)), 2)}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1312_3426_gb300 import build as lbuild
    from paper_1312_3426_gb300 import lbib
    if rank == 0:
        lbuild.build()
    if world > 1:
        dist.barrier()
    lbib.load()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    if args.workload == "batch64":
        scs, cells, nodes, ms, clocks, tuned = batch_workload(args, lbib, torch, dev, stream)
        ms = max_over_ranks(ms, dev)
        peak, peak_kind = measured_peak()
        bpc = BYTES_PER_CELL[args.precision]
        achieved = bpc * cells / (ms / args.steps / 1e3) / 1e9
        if rank == 0:
            line = {
                "metric": METRIC, "value": round(whole_job_mlups(cells, args.steps, ms, world), 2), "unit": "MLUPS",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic (seeded batch of channels)",
                "config": {"workload": f"batch_mix: {len(scs)} channels, boxes 32^3..128x64x64, "
                                       f"{sum(len(x.objects) for x in scs)} cells (levels 2-4), {nodes} nodes, "
                                       f"{cells} fluid cells", "tuning": tuned,
                           "l2": "inputs larger than L2, no flush",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 4), "traffic": None,
                             "kernel": "whole batched step (all kernels)", "bytes_per_cell": bpc,
                             "peak_source": peak_kind + " copy bandwidth"},
                "nodes_per_s": round(world * nodes * args.steps / (ms / 1e3), 1),
                # per step: fluid, node and membrane launches; the counter
                # advance per 16-step graph; every 128 steps one mask-rebuild
                # launch per channel with cells
                "gpu_launches": args.steps * 3 + args.steps // 16
                + (args.steps // 128) * sum(1 for x in scs if x.objects),
                "clocks": clocks, "e2e": None, "cpu_baseline": None,
            }
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    sc = make_scene(args.workload)
    peak, peak_kind = measured_peak()
    m = measure(args, lbib, torch, sc, args.precision, stream, dev, local, world, barrier, e2e=not args.no_e2e,
                launch=args.launch, clocks=True)
    ms, value, nf, bpc = m["ms"], m["value"], sc.n_fluid_cells, BYTES_PER_CELL[args.precision]
    fluid_ms, nodes_ms, membrane_ms = m["fluid_ms"], m["nodes_ms"], m["membrane_ms"]
    achieved = bpc * nf / (fluid_ms / 1e3) / 1e9
    traffic = profiled_traffic(args.workload, args.precision, nf)
    clocks, e2e, persistent = m["clocks"], m["e2e"], args.launch == "batched"

    precision = None
    if not args.no_precision:
        precision = precision_records(args, lbib, torch, stream, dev, local, world, barrier, peak, m)

    serving = None
    if world == 1 and not args.no_serving:
        serving = serving_comparison(args, stream.cuda_stream)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(sc, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision if args.precision != "f32" else "f32",
            "data": "synthetic (seeded channel, Evans-Fung RBC meshes at random non-overlapping poses)",
            "config": {"workload": workload_desc(sc), "precision_storage": args.precision,
                       "fluid_cells": nf, "nodes": sc.n_nodes, "objects": len(sc.objects),
                       "l2": "inputs larger than L2 (populations %.0f MB), no flush" % (bpc * nf / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU", "tuning": m["tuning"]},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "kernel": f"k_batch_fluid<{args.precision}>" if persistent else f"{m['kernel']}<{args.precision}>",
                         "bytes_per_cell": bpc, "mean_launch_ms": round(fluid_ms, 5),
                         "launches_timed": m["fluid_launches"], "peak_source": peak_kind + " copy bandwidth"},
            "step_breakdown_ms": {"fluid": round(fluid_ms, 5), "nodes": round(nodes_ms, 5),
                                  "membrane_overlapped": round(membrane_ms, 5)},
            "nodes_per_s": round(world * sc.n_nodes * args.steps / (ms / 1e3), 1),
            "step_hbm_frac": round((bpc * nf + 400 * sc.n_nodes) / (ms / args.steps / 1e3) / 1e9 / peak, 4),
            # per step: fluid, node update and (second stream) membrane
            # kernels; the active-cell mask is rebuilt every 128 steps
            "gpu_launches": args.steps * (3 if sc.objects else 1) + (args.steps // 16 if persistent else 0)
            + (args.steps // 128 if sc.objects else 0),
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": base,
            "precision": precision,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
