"""The autotuner's search space (paper_1312_3426_gb300/tune.py), on the host
with stand-in simulations: which knob groups it searches for which
workloads, that every candidate is a valid knob setting, and that the
search keeps the fastest candidate of each group given the groups before it."""
import pytest

from paper_1312_3426_gb300 import lbib, tune


class FakeSim:
    """info(): n_templates, n_objects, n_nodes, cells, steps, bytes, precision, kernel."""

    def __init__(self, objects, prec, cost):
        self._info = [1, objects, 642 * objects, 1 << 20, 0, 0, prec, 0]
        self.h = self
        self.knobs = {}
        self.cost = cost

    def info(self):
        return self._info


@pytest.fixture
def fake_lbib(monkeypatch):
    def set_tuning(h, key, value):
        h.knobs[key] = value
    monkeypatch.setattr(lbib, "lbib_set_tuning", set_tuning)
    tune._CACHE.clear()
    yield
    tune._CACHE.clear()


def names_of(groups):
    return [names for names, _ in groups]


def test_search_groups_by_workload(fake_lbib):
    f32 = [FakeSim(200, lbib.LBIB_POP_F32, None)]
    f16 = [FakeSim(200, lbib.LBIB_POP_F16S, None)]
    free = [FakeSim(0, lbib.LBIB_POP_F16S, None)]
    assert names_of(tune.candidates(f32, False)) == [("cluster", "overlap"), ("membrane_threads", "membrane_group"),
                                                     ("node_threads",), ("early_launch",)]
    assert ("fluid_kernel",) in names_of(tune.candidates(f16, False))
    assert names_of(tune.candidates(free, False)) == [("fluid_kernel",), ("early_launch",)]
    batched = names_of(tune.candidates(f16 * 3, True))
    assert ("early_launch",) not in batched and ("fluid_kernel",) in batched
    for names, values in tune.candidates(f16, False):
        for vals in values:
            knobs = dict(zip(names, vals))
            if "membrane_threads" in knobs:
                t, g = knobs["membrane_threads"], knobs["membrane_group"]
                assert t % 32 == 0 and 32 <= t <= 256 and 1 <= g <= 15 and t * g <= 1024
            if "fluid_kernel" in knobs:
                assert knobs["fluid_kernel"] in (1, 2, 3)
    assert any(v == (128, 5) for names, values in tune.candidates(f32, False) for v in values
               if names == ("membrane_threads", "membrane_group"))


def test_autotune_keeps_the_fastest_of_each_group(fake_lbib, monkeypatch):
    """With a synthetic cost that is lowest at threads 128, 5 objects per
    block, 64-node chunks and early launch on, the search finds exactly
    that, applies it to every simulation and caches it by workload class."""
    best = {"membrane_threads": 128, "membrane_group": 5, "node_threads": 64, "early_launch": 1}
    key_of = dict((key, name) for name, key in tune.KNOBS)

    def cost(sims, steps, batched):
        knobs = {key_of[k]: v for k, v in sims[0].knobs.items()}
        return 1.0 + sum(abs(knobs[n] - v) for n, v in best.items()) + 0.5 * knobs["cluster"]

    monkeypatch.setattr(tune, "_time", cost)
    sims = [FakeSim(200, lbib.LBIB_POP_F32, None)]
    choice, timing = tune.autotune(sims, steps=8)
    for n, v in best.items():
        assert choice[n] == v
    assert choice["cluster"] == 1
    assert {key_of[k]: v for k, v in sims[0].knobs.items()} == choice
    assert len(timing) == sum(len(v) for _, v in tune.candidates(sims, False))
    again, _ = tune.autotune([FakeSim(200, lbib.LBIB_POP_F32, None)], steps=8)
    assert again == choice
