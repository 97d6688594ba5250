"""Slab decomposition of one domain along its march axis (z in 3D, y in 2D).

MacLAB is a radius-1 stencil: every velocity c_a of Eqs. (4)-(5) moves at most
one node along each axis, so a node's update reads only the planes next to
its own.  A domain split into slabs along the march axis therefore needs ghost
planes beside every slab, refreshed from the neighbouring slabs.  A slab is an
ordinary domain of the library, closed along the axis: its outermost plane on
each side is a wall plane (the step kernels never write walls: the paper
retains wall values with no calculation, Tests 1-3 and 5) and the next
depth - 1 planes are fluid copies of the neighbour's planes.  After every
exchange all those planes hold the neighbour's values; each step spoils one
more plane from each end (the wall plane does not advance), so with depth h
the interior stays exact for h steps and the exchange of h planes per side
follows every h steps (depth 1: one wall plane, exchanged every step).  Every
interior node thus sees exactly the upstream values of the undivided domain,
and the slabs' interiors equal the undivided run bit for bit.

This module holds no arithmetic of the method: partitioning, ghost-plane
bookkeeping and the exchange pattern.  The stepping is done by a "stepper"
(the library's Solver, one per slab), the copies by a "transport": copies
between slabs of one process (``SlabDomain``) or messages between ranks of
``torch.distributed`` (``DistributedSlab``: NCCL between GPUs, gloo in the CPU
tests).  Diagnostics are the raw FP64 sums of ``maclab_diagnostics_sums``
added over slabs (an all-reduce across ranks).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs


def partition(n_planes: int, n_slabs: int):
    """Balanced [start, stop) plane ranges of n_slabs slabs (n_slabs <= n_planes)."""
    if n_slabs < 1 or n_slabs > n_planes:
        raise ValueError(f"cannot split {n_planes} planes into {n_slabs} slabs")
    bounds = [(n_planes * i) // n_slabs for i in range(n_slabs + 1)]
    return [(bounds[i], bounds[i + 1]) for i in range(n_slabs)]


def _axis_bit(case) -> int:
    return 0b100 if case.d == 3 else 0b010


def slab_case(case: inputs.Case, start: int, stop: int, depth: int = 1) -> inputs.Case:
    """The slab of planes [start, stop) with `depth` ghost planes on each side.

    The outermost ghost plane on each side is made of wall nodes of an extra
    wall id (its table values are placeholders: the exchange overwrites the
    ghosts before the first step); the others keep the node types of the
    planes they copy.  Ghosts start as copies of the neighbouring planes
    (wrapped on a periodic axis; on a closed axis the outer plane of the domain
    is a wall that no fluid node reads past, and the ghosts copy it).  The
    slab is closed along the axis.
    """
    if depth < 1:
        raise ValueError("depth must be >= 1")
    n = case.grid[0]
    periodic_axis = bool(case.periodic & _axis_bit(case))
    idx = np.arange(start - depth, stop + depth)
    if periodic_axis:
        idx = idx % n
    else:
        idx = np.clip(idx, 0, n - 1)
    rho = case.rho[idx].copy()
    u = case.u[:, idx].copy()
    d = case.d
    if case.node_type is None:
        nt = np.zeros(rho.shape, dtype=np.uint8)
        wall_rho = np.zeros(0)
        wall_u = np.zeros((0, d))
    else:
        nt = case.node_type[idx].copy()
        wall_rho = np.asarray(case.wall_rho, dtype=np.float64)
        wall_u = np.asarray(case.wall_u, dtype=np.float64).reshape(-1, d)
    ghost_id = len(wall_rho) + 1
    if ghost_id > 255:
        raise ValueError("no wall id left for the ghost planes")
    nt[0] = ghost_id
    nt[-1] = ghost_id
    wall_rho = np.concatenate([wall_rho, [1.0]])
    wall_u = np.concatenate([wall_u, np.zeros((1, d))])
    dims = case.dims[:-1] + (stop - start + 2 * depth,)
    return inputs.Case(case.lattice, dims, case.periodic & ~_axis_bit(case), rho, u, nt, wall_rho,
                       wall_u, force=case.force, name=f"{case.name}-slab{start}-{stop}")


@dataclasses.dataclass
class _Slab:
    start: int
    stop: int
    solver: object
    depth: int = 1

    @property
    def planes(self):
        return self.stop - self.start


def _neighbours(i, k, periodic_axis):
    lo = (i - 1) % k if (periodic_axis or i > 0) else None
    hi = (i + 1) % k if (periodic_axis or i < k - 1) else None
    return lo, hi


def combine_sums(sums, n_fluid, rho0=1.0, e=1.0):
    """maclab_diagnostics-style values from raw sums added over slabs."""
    s = np.asarray(sums, dtype=np.float64)
    out = {"mass": rho0 * (n_fluid + s[0]), "kinetic": 0.5 * rho0 * e * e * s[1],
           "momentum": list(rho0 * e * s[2:5]), "max_u_lattice": float(s[7]), "nonfinite": int(s[8])}
    out["residual"] = float(np.sqrt(s[5] / s[6])) if s[5] >= 0 and s[6] > 0 else -1.0
    return out


class SlabDomain:
    """One domain as k slabs stepped in one process (one GPU or several),
    ghost planes exchanged through device buffers after every step."""

    def __init__(self, case: inputs.Case, k: int, precision, devices=None, kernel=None, depth=1):
        import torch

        from . import maclab as M
        self.M, self.torch = M, torch
        self.case = case
        self.k = k
        self.periodic_axis = bool(case.periodic & _axis_bit(case))
        self.depth = depth
        self.slabs = []
        for i, (a, b) in enumerate(partition(case.grid[0], k)):
            if b - a < depth:
                raise ValueError("every slab needs at least `depth` planes")
            dev = devices[i % len(devices)] if devices else torch.cuda.current_device()
            with torch.cuda.device(dev):
                sub = slab_case(case, a, b, depth)
                s = M.Solver.from_case(sub, precision)
                if kernel is not None:
                    s.set_kernel(kernel)
            self.slabs.append(_Slab(a, b, s, depth))
        self._bufs = {}
        self.exchange()

    def _buf(self, slab):
        s = slab.solver
        key = id(s)
        if key not in self._bufs:
            plane = s.state_bytes() // (slab.planes + 2 * self.depth)
            self._bufs[key] = self.torch.empty(plane * self.depth, dtype=self.torch.uint8, device="cuda")
        return self._bufs[key]

    def exchange(self):
        """Ghost planes [0, h) of slab i <- the last h interior planes of slab i - 1;
        ghost planes [h + P, 2h + P) <- the first h interior planes of slab i + 1
        (wrapped on a periodic axis); h = depth, P = the slab's interior planes."""
        M, h = self.M, self.depth
        for i, sl in enumerate(self.slabs):
            lo, hi = _neighbours(i, self.k, self.periodic_axis)
            if lo is not None:
                src = self.slabs[lo]
                buf = self._buf(src)
                M.maclab_get_planes(src.solver.handle, src.planes, h, buf)
                src.solver.sync()
                M.maclab_set_planes(sl.solver.handle, 0, h, buf)
                sl.solver.sync()
            if hi is not None:
                src = self.slabs[hi]
                buf = self._buf(src)
                M.maclab_get_planes(src.solver.handle, h, h, buf)
                src.solver.sync()
                M.maclab_set_planes(sl.solver.handle, h + sl.planes, h, buf)
                sl.solver.sync()

    def step(self, n=1):
        """n steps: runs of `depth` steps per slab, each followed by an exchange."""
        left = int(n)
        while left > 0:
            k = min(self.depth, left)
            for sl in self.slabs:
                sl.solver.step(k)
            self.exchange()
            left -= k

    def get_state(self):
        """Physical (rho, u) of the whole domain, assembled from the interiors."""
        rho = np.empty(self.case.grid)
        u = np.empty((self.case.d,) + self.case.grid)
        h = self.depth
        for sl in self.slabs:
            r, v = sl.solver.get_state()
            rho[sl.start:sl.stop] = r[h:h + sl.planes]
            u[:, sl.start:sl.stop] = v[:, h:h + sl.planes]
        return rho, u

    def diagnostics(self):
        """Sums over every slab's fluid nodes (depth 1: exactly the domain's)."""
        if self.depth != 1:
            raise ValueError("diagnostics over slabs need depth 1 (fluid halo planes would count twice)")
        tot = np.zeros(9)
        for sl in self.slabs:
            s = self.M.maclab_diagnostics_sums(sl.solver.handle)
            tot[[0, 1, 2, 3, 4, 8]] += np.asarray(s)[[0, 1, 2, 3, 4, 8]]
            tot[5] = -1.0 if s[5] < 0 or tot[5] < 0 else tot[5] + s[5]
            tot[6] = -1.0 if s[6] < 0 or tot[6] < 0 else tot[6] + s[6]
            tot[7] = max(tot[7], s[7])
        return combine_sums(tot, self.case.n_fluid)

    def close(self):
        for sl in self.slabs:
            sl.solver.close()


class DistributedSlab:
    """This rank's slab of a domain split over the ranks of torch.distributed.

    ``stepper`` advances the slab (``step(n)``) and moves raw planes
    (``get_planes(p0, count) -> tensor``, ``set_planes(p0, count, tensor)``);
    the exchange sends this slab's edge planes to the neighbouring ranks and
    receives their edge planes into the ghost planes, every step.  With the
    library's Solver as stepper the planes are device tensors moved by NCCL;
    the CPU tests use the FP64 oracle as stepper with host tensors over gloo.
    """

    def __init__(self, case: inputs.Case, stepper_factory, rank=None, world=None, depth=1):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank() if rank is None else rank
        self.world = dist.get_world_size() if world is None else world
        self.case = case
        self.periodic_axis = bool(case.periodic & _axis_bit(case))
        self.start, self.stop = partition(case.grid[0], self.world)[self.rank]
        self.depth = depth
        self.planes = self.stop - self.start
        if self.planes < depth:
            raise ValueError("every slab needs at least `depth` planes")
        self.sub = slab_case(case, self.start, self.stop, depth)
        self.stepper = stepper_factory(self.sub)
        self.exchange()

    def exchange(self):
        import torch
        dist = self.dist
        lo, hi = _neighbours(self.rank, self.world, self.periodic_axis)
        h = self.depth
        send_lo = self.stepper.get_planes(h, h) if lo is not None else None
        send_hi = self.stepper.get_planes(self.planes, h) if hi is not None else None
        recv_lo = torch.empty_like(send_lo if send_lo is not None else send_hi) if lo is not None else None
        recv_hi = torch.empty_like(send_hi if send_hi is not None else send_lo) if hi is not None else None
        # Messages between two ranks are matched in the order they are posted
        # (NCCL has no tags), and on a periodic axis with two ranks the lower and
        # upper neighbour are the same rank.  So every rank posts its sends in the
        # order (to lo: first plane, to hi: last plane) and its receives in the
        # order (from hi, from lo): the k-th message a rank sends to a peer is then
        # the k-th it receives from that peer.
        ops = []
        if lo is not None:
            ops.append(dist.P2POp(dist.isend, send_lo, lo))
        if hi is not None:
            ops.append(dist.P2POp(dist.isend, send_hi, hi))
        if hi is not None:
            ops.append(dist.P2POp(dist.irecv, recv_hi, hi))
        if lo is not None:
            ops.append(dist.P2POp(dist.irecv, recv_lo, lo))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        if lo is not None:
            self.stepper.set_planes(0, h, recv_lo)
        if hi is not None:
            self.stepper.set_planes(h + self.planes, h, recv_hi)

    def step(self, n=1):
        """n steps: runs of `depth` steps, each followed by an exchange."""
        left = int(n)
        while left > 0:
            k = min(self.depth, left)
            self.stepper.step(k)
            self.exchange()
            left -= k

    def interior(self):
        """This rank's interior planes of (rho, u) (stepper units)."""
        r, v = self.stepper.get_state()
        h = self.depth
        return r[h:h + self.planes], v[:, h:h + self.planes]


class SolverStepper:
    """The library's Solver as a DistributedSlab stepper (device planes, NCCL)."""

    def __init__(self, sub: inputs.Case, precision, kernel=None):
        import torch

        from . import maclab as M
        self.M, self.torch = M, torch
        self.solver = M.Solver.from_case(sub, precision)
        if kernel is not None:
            self.solver.set_kernel(kernel)
        self.plane_bytes = self.solver.state_bytes() // sub.grid[0]

    def step(self, n):
        self.solver.step(n)

    def get_planes(self, p0, count):
        buf = self.torch.empty(self.plane_bytes * count, dtype=self.torch.uint8, device="cuda")
        self.M.maclab_get_planes(self.solver.handle, p0, count, buf)
        self.solver.sync()
        return buf

    def set_planes(self, p0, count, buf):
        self.M.maclab_set_planes(self.solver.handle, p0, count, buf)
        self.solver.sync()

    def get_state(self):
        return self.solver.get_state()

    def diagnostics_sums(self):
        return self.M.maclab_diagnostics_sums(self.solver.handle)
