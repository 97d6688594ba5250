"""Slab decomposition along the march axis: host logic on the CPU.

* partitioning and the slab domains (ghost planes, wall ids, periodicity);
* two gloo ranks, each stepping its slab with the FP64 oracle and exchanging
  ghost planes every step through torch.distributed: the interiors equal the
  undivided oracle run bit for bit (a radius-1 stencil sees the same upstream
  values), for a periodic Taylor-Green field, a lid-driven cavity and a 2D
  channel.
The GPU form (slabs of the CUDA library exchanging through device buffers) is
tested in test_slabs_gpu.py.
"""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs, slabs


def test_partition_is_balanced_and_complete():
    for n, k in ((128, 2), (10, 3), (7, 7), (1000, 8)):
        p = slabs.partition(n, k)
        assert p[0][0] == 0 and p[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
        sizes = [b - a for a, b in p]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slabs.partition(3, 4)


def test_slab_case_ghost_planes():
    case = inputs.cavity3d(12, lid=0.05)
    sub = slabs.slab_case(case, 4, 8)
    assert sub.dims == (12, 12, 6) and sub.periodic == 0
    ghost = len(case.wall_rho) + 1
    assert np.all(sub.node_type[0] == ghost) and np.all(sub.node_type[-1] == ghost)
    assert np.array_equal(sub.node_type[1:-1], case.node_type[4:8])
    tg = inputs.tgv3d(8, 0.02)
    sub = slabs.slab_case(tg, 0, 4)
    assert sub.periodic == 0b011
    assert np.array_equal(sub.u[:, 0], tg.u[:, 7])         # wrapped lower ghost
    assert np.array_equal(sub.u[:, -1], tg.u[:, 4])
    sub = slabs.slab_case(tg, 0, 4, depth=3)
    assert sub.dims == (8, 8, 10)
    assert np.all(sub.node_type[0] == 1) and np.all(sub.node_type[1:-1] == 0)
    assert np.array_equal(sub.u[:, :3], tg.u[:, 5:8])      # wrapped: planes 5, 6, 7


class OracleStepper:
    """The FP64 oracle on one slab (lattice units): planes as host tensors."""

    def __init__(self, sub):
        self.sub = sub
        self.rho, self.u = sub.rho.copy(), sub.u.copy()

    def step(self, n):
        self.rho, self.u = orc.step(self.sub.lattice, self.rho, self.u, self.sub.periodic,
                                    wall=self.sub.wall_mask, force=self.sub.force, nsteps=n)

    def get_planes(self, p0, count):
        import torch
        return torch.from_numpy(np.concatenate([self.rho[None, p0:p0 + count],
                                                self.u[:, p0:p0 + count]]).copy())

    def set_planes(self, p0, count, buf):
        a = buf.numpy()
        self.rho[p0:p0 + count] = a[0]
        self.u[:, p0:p0 + count] = a[1:]

    def get_state(self):
        return self.rho, self.u


def _rank(rank, world, port, name, depth, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case, steps = _case(name)
        sl = slabs.DistributedSlab(case, OracleStepper, depth=depth)
        sl.step(steps)
        r, u = sl.interior()
        q.put((rank, sl.start, sl.stop, r, u))
    finally:
        dist.destroy_process_group()


def _case(name):
    if name == "tgv3d":
        return inputs.tgv3d(12, 0.05, noise_sigma=1e-3, seed=3), 6
    if name == "cavity3d":
        return inputs.cavity3d(12, lid=0.1), 6
    return inputs.channel2d(nx=10, ny=17, u_top=0.1, force_x=1e-4), 8


@pytest.mark.parametrize("name,depth", [("tgv3d", 1), ("cavity3d", 1), ("channel2d", 1),
                                        ("tgv3d", 3), ("channel2d", 4)])
def test_two_gloo_ranks_equal_undivided_run(name, depth):
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, name, depth, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case, steps = _case(name)
    r_ref, u_ref = orc.step(case.lattice, case.rho, case.u, case.periodic, wall=case.wall_mask,
                            force=case.force, nsteps=steps)
    for rank, a, b, r, u in got:
        assert np.array_equal(r, r_ref[a:b]), (name, rank)
        assert np.array_equal(u, u_ref[:, a:b]), (name, rank)
