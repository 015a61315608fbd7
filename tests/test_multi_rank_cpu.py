"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2):
replicas are timed by the slowest rank and the job's value is the sum over
ranks.  No GPU is touched."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 10.0 + 5.0 * rank            # rank 1 is the slower replica
        ms = bench.max_over_ranks(ms_local)
        value = bench.whole_job_mlups(1_000_000, 100, ms, world)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_replicas_timed_by_slowest_rank_and_summed():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    ms_expected = 15.0
    value_expected = world * 1_000_000 * 100 / (ms_expected / 1e3) / 1e6
    assert res[0] == res[1] == (ms_expected, pytest.approx(value_expected))


def test_single_rank_has_no_reduction():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_mlups(10, 4, 2.0, 1) == pytest.approx(10 * 4 / 2e-3 / 1e6)
