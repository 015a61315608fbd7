"""Autotuner for the launch-shape knobs of the C ABI.

The knobs (``lbib_set_tuning``) change no result beyond the order of
floating-point atomics, only the speed: the thread blocks per object of the
membrane-force kernel (``LBIB_TUNE_IB_CLUSTER``), its block size
(``LBIB_TUNE_MEMBRANE_THREADS``) and whether that kernel overlaps the fluid
kernel on a second stream (``LBIB_TUNE_OVERLAP``).
``autotune`` times a few steps of the caller's own simulations for each
candidate and keeps the fastest; results are cached by a key of the
workload's shape (box-size class, storage precision, largest template), so
simulations of the same class reuse the choice.  Tuning advances the
simulations it times; callers tune on a throw-away copy or accept the steps.
"""
from __future__ import annotations

import time

from . import lbib

_CACHE: dict = {}


def _key(sims):
    infos = [s.info() for s in sims]
    cells = sum(int(i[3]) for i in infos)
    nodes = sum(int(i[2]) for i in infos)
    prec = sorted({int(i[6]) for i in infos})
    cls = lambda v: 0 if v <= 0 else int(round(float(v) ** 0.5).bit_length())  # noqa: E731
    return (len(sims), cls(cells), cls(nodes), tuple(prec))


def _time(sims, steps, batched):
    if batched:
        lbib.lbib_batch_step([s.h for s in sims], steps)
    else:
        for s in sims:
            s.step(steps)
        for s in sims:
            s.sync()
    t0 = time.perf_counter()
    if batched:
        lbib.lbib_batch_step([s.h for s in sims], steps)
    else:
        for s in sims:
            s.step(steps)
        for s in sims:
            s.sync()
    return time.perf_counter() - t0


def autotune(sims, clusters=(1, 2), overlaps=(1, 0), threads=(192, 256), steps=32, batched=None):
    """Chooses and applies the fastest (cluster, overlap, membrane threads)
    for `sims` (Sim objects); returns the choice and the measured seconds
    per candidate."""
    sims = list(sims)
    if batched is None:
        batched = len(sims) > 1
    key = _key(sims) + (batched,)
    if key in _CACHE:
        best = _CACHE[key][0]
        _apply(sims, *best)
        return _CACHE[key]
    if not any(s.obj_tid for s in sims):
        best, timing = (1, 1, 192), {}
    else:
        timing = {}
        for c in clusters:
            for ov in overlaps:
                for th in threads:
                    _apply(sims, c, ov, th)
                    timing[(c, ov, th)] = _time(sims, steps, batched)
        best = min(timing, key=timing.get)
    _apply(sims, *best)
    _CACHE[key] = (best, timing)
    return _CACHE[key]


def _apply(sims, cluster, overlap, threads=192):
    for s in sims:
        lbib.lbib_set_tuning(s.h, lbib.LBIB_TUNE_IB_CLUSTER, cluster)
        lbib.lbib_set_tuning(s.h, lbib.LBIB_TUNE_OVERLAP, overlap)
        lbib.lbib_set_tuning(s.h, lbib.LBIB_TUNE_MEMBRANE_THREADS, threads)
