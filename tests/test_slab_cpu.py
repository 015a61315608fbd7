"""Slab decomposition along x on CPU ranks (gloo): each rank steps the FP64
oracle on its slab plus two ghost planes and exchanges the ghost planes with
its neighbours before every step; the interiors after the steps equal the
undecomposed run exactly.  The halo bookkeeping is paper_1312_3426_gb300.slab.
No GPU is touched."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NX, NY, NZ, STEPS = 13, 9, 5, 12
PARAMS = dict(walls=True, tau=0.8, rho0=1.0, body_force=(2e-5, 0.0, 1e-5))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _initial_state(e, w):
    """Equilibrium populations [nz][ny][nx][19] of a density and velocity
    field that vary along x (so that the slab faces matter)."""
    z, y, x = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    rho = 1.0 + 0.01 * np.sin(2 * np.pi * x / NX)
    u = np.stack([0.02 * np.sin(2 * np.pi * (x / NX + z / NZ)),
                  0.005 * np.cos(2 * np.pi * x / NX) * np.sin(np.pi * y / (NY - 1)),
                  0.01 * np.cos(2 * np.pi * (x / NX - y / NY))], axis=-1)
    eu = np.einsum("zyxk,qk->zyxq", u, e.astype(np.float64))
    usq = np.sum(u * u, axis=-1)[..., None]
    return w * rho[..., None] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq)


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1312_3426_gb300 import slab
        x0, x1 = slab.slab_bounds(NX, rank, world)
        n = x1 - x0
        left, right = slab.neighbours(rank, world)
        full0 = oracle.Oracle(NX, NY, NZ, **PARAMS)
        e, w = full0.lattice()
        f0 = _initial_state(e, w)
        loc = oracle.Oracle(n + 2, NY, NZ, **PARAMS)
        loc.set_populations(slab.ghosted(f0, NX, rank, world, axis=2))
        for _ in range(STEPS):
            f = loc.populations()
            # my first plane goes to the left neighbour's right ghost, my last
            # plane to the right neighbour's left ghost (tags: 0 leftwards, 1 rightwards)
            send_l = torch.from_numpy(np.ascontiguousarray(f[:, :, 1, :]))
            send_r = torch.from_numpy(np.ascontiguousarray(f[:, :, n, :]))
            recv_l = torch.empty_like(send_l)  # left neighbour's last plane -> my left ghost
            recv_r = torch.empty_like(send_r)  # right neighbour's first plane -> my right ghost
            reqs = [dist.isend(send_l, left, tag=0), dist.isend(send_r, right, tag=1),
                    dist.irecv(recv_l, left, tag=1), dist.irecv(recv_r, right, tag=0)]
            for r in reqs:
                r.wait()
            f[:, :, 0, :] = recv_l.numpy()
            f[:, :, n + 1, :] = recv_r.numpy()
            loc.set_populations(f)
            loc.step(1)
        mine = loc.populations()[:, :, 1:n + 1, :]
        full0.set_populations(f0)
        full0.step(STEPS)
        ref = full0.populations()[:, :, x0:x1, :]
        out[rank] = (bool(np.array_equal(mine, ref)), float(np.abs(mine - ref).max()),
                     float(np.abs(ref - f0[:, :, x0:x1, :]).max()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_decomposition_equals_the_whole_box(world):
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        equal, diff, moved = res[rank]
        assert moved > 1e-6          # the state did change over the steps
        assert equal, (rank, diff)


def test_slab_bookkeeping():
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1312_3426_gb300 import slab
    for nx, world in ((13, 2), (13, 3), (7, 7), (256, 8)):
        spans = [slab.slab_bounds(nx, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == nx
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
        for r in range(world):
            gl, gr = slab.ghost_sources(nx, r, world)
            left, right = slab.neighbours(r, world)
            assert gl == spans[left][1] - 1 and gr == spans[right][0]
    with pytest.raises(ValueError):
        slab.slab_bounds(3, 0, 4)
    e, _ = oracle.Oracle(4, 4, 4).lattice()
    from_left, from_right = slab.crossing_directions(e)
    assert len(from_left) == 5 and len(from_right) == 5
    assert all(e[q][0] == 1 for q in from_left) and all(e[q][0] == -1 for q in from_right)
