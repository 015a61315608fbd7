"""Autotuner for the launch-shape knobs of the C ABI.

The knobs (``lbib_set_tuning``) change no result beyond the order of
floating-point atomics, only the speed:

* ``LBIB_TUNE_IB_CLUSTER``      thread blocks per object of the membrane kernel;
* ``LBIB_TUNE_OVERLAP``         membrane kernel beside the fluid kernel (second stream);
* ``LBIB_TUNE_MEMBRANE_THREADS`` threads per object of the membrane kernel;
* ``LBIB_TUNE_MEMBRANE_GROUP``  objects per block of the membrane kernel;
* ``LBIB_TUNE_NODE_THREADS``    nodes per block of the node kernel (the node chunk);
* ``LBIB_TUNE_FLUID_KERNEL``    16-bit storage: two cells per thread (1), the
  warp-specialised two-cells kernel (2, single simulations only) or one
  cell per thread (3);
* ``LBIB_TUNE_EARLY_LAUNCH``    programmatic dependent launch of the node and
  fluid kernels (single simulations).

``autotune`` times a few steps of the caller's own simulations for each
candidate and keeps the fastest, one knob group at a time (membrane
clusters and overlap, then threads per object together with objects per
membrane block, then the node chunk, then the fluid kernel, then early
launch, each group searched with the best choice of the groups before it).  Results are cached by a key of
the workload's shape (number of simulations, box-size class, node-count
class, storage precisions, batched or not), so simulations of the same class
reuse the choice.  Tuning advances the simulations it times; callers tune on
a throw-away copy or accept the steps.
"""
from __future__ import annotations

import time

from . import lbib

_CACHE: dict = {}

KNOBS = (("cluster", lbib.LBIB_TUNE_IB_CLUSTER), ("overlap", lbib.LBIB_TUNE_OVERLAP),
         ("membrane_threads", lbib.LBIB_TUNE_MEMBRANE_THREADS), ("membrane_group", lbib.LBIB_TUNE_MEMBRANE_GROUP),
         ("node_threads", lbib.LBIB_TUNE_NODE_THREADS), ("fluid_kernel", lbib.LBIB_TUNE_FLUID_KERNEL),
         ("early_launch", lbib.LBIB_TUNE_EARLY_LAUNCH))
DEFAULT = {"cluster": 1, "overlap": 1, "membrane_threads": 192, "membrane_group": 1, "node_threads": 256,
           "fluid_kernel": 0, "early_launch": 0}


def _key(sims, batched):
    infos = [s.info() for s in sims]
    cells = sum(int(i[3]) for i in infos)
    nodes = sum(int(i[2]) for i in infos)
    prec = sorted({int(i[6]) for i in infos})
    cls = lambda v: 0 if v <= 0 else int(round(float(v) ** 0.5).bit_length())  # noqa: E731
    return (len(sims), cls(cells), cls(nodes), tuple(prec), bool(batched))


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


def apply(sims, choice):
    """Sets every knob of `choice` (a dict with the keys of DEFAULT)."""
    for s in sims:
        for name, key in KNOBS:
            lbib.lbib_set_tuning(s.h, key, int(choice[name]))


def candidates(sims, batched, clusters=(1, 2), overlaps=(1, 0), threads=(96, 128, 192, 256),
               member_groups=(1, 2, 3, 4, 5, 6), node_threads=(64, 128, 256)):
    """The knob groups searched, in order: [(name, ...), [values, ...]].
    Threads per object and objects per block are searched together: fewer
    threads leave more of each SM to the fluid kernel beside the membrane
    kernel until the membrane kernel becomes the longer of the two, and
    where that happens depends on how many objects share a block."""
    groups = []
    has_objects = any(int(s.info()[1]) > 0 for s in sims)
    if has_objects:
        groups.append((("cluster", "overlap"), [(c, o) for c in clusters for o in overlaps]))
        groups.append((("membrane_threads", "membrane_group"),
                       [(t, g) for t in threads for g in member_groups if t * g <= 1024]))
        groups.append((("node_threads",), [(t,) for t in node_threads]))
    if any(int(s.info()[6]) != lbib.LBIB_POP_F32 for s in sims):
        kernels = (1, 3) if batched else (1, 2, 3)
        groups.append((("fluid_kernel",), [(k,) for k in kernels]))
    if not batched:  # the batched step launches plainly
        groups.append((("early_launch",), [(0,), (1,)]))
    return groups


def autotune(sims, steps=32, batched=None, **search):
    """Chooses and applies the fastest knobs for `sims` (Sim objects);
    returns (choice, seconds per candidate): choice is a dict with the keys
    of DEFAULT, the timing dict is keyed by 'name=value,...' strings."""
    sims = list(sims)
    if batched is None:
        batched = len(sims) > 1
    key = _key(sims, batched)
    if key in _CACHE:
        apply(sims, _CACHE[key][0])
        return _CACHE[key]
    best = dict(DEFAULT)
    timing = {}
    for names, values in candidates(sims, batched, **search):
        group_t = {}
        for vals in values:
            trial = dict(best, **dict(zip(names, vals)))
            apply(sims, trial)
            t = _time(sims, steps, batched)
            group_t[vals] = t
            timing[",".join(f"{n}={v}" for n, v in zip(names, vals))] = t
        best.update(dict(zip(names, min(group_t, key=group_t.get))))
    apply(sims, best)
    _CACHE[key] = (best, timing)
    return _CACHE[key]
