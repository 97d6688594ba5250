"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: only initial fields, node-type
masks and wall tables for the flows the paper runs (Couette and
Couette-Poiseuille, Tests 1-2; lid-driven cavities, Tests 3 and 5; Taylor-Green
vortex, Test 4), plus random fields for parity checks.  Velocities are in
lattice units (u / e) unless a name says otherwise.  Array axes are [y, x] in
2D and [z, y, x] in 3D, x fastest; a velocity field is [d, *grid].

Node types: 0 = fluid, k >= 1 = wall id k, whose (rho, u) come from the wall
tables (row k - 1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 190102716
D2Q9, D3Q19 = 0, 1


def rng(seed_offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + seed_offset))


@dataclasses.dataclass
class Case:
    """One flow set-up in lattice units."""
    lattice: int
    dims: tuple            # (nx, ny) or (nx, ny, nz)
    periodic: int          # bit0 x, bit1 y, bit2 z
    rho: np.ndarray        # [*grid], rho / rho0
    u: np.ndarray          # [d, *grid], u / e
    node_type: np.ndarray | None = None   # uint8 [*grid] or None (all fluid)
    wall_rho: np.ndarray | None = None    # [n_wall_ids]
    wall_u: np.ndarray | None = None      # [n_wall_ids, d]
    force: tuple | None = None            # lattice-unit increment per step
    name: str = ""

    @property
    def d(self) -> int:
        return 2 if self.lattice == D2Q9 else 3

    @property
    def grid(self) -> tuple:
        return tuple(reversed(self.dims))

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.dims))

    @property
    def n_fluid(self) -> int:
        return self.n_nodes if self.node_type is None else int(np.sum(self.node_type == 0))

    @property
    def wall_mask(self):
        return None if self.node_type is None else (self.node_type != 0)


def place_walls(rho, u, node_type, wall_rho, wall_u):
    """Write each wall id's tabulated (rho, u) into the wall nodes (assignment only)."""
    rho = np.array(rho, dtype=np.float64, copy=True)
    u = np.array(u, dtype=np.float64, copy=True)
    if node_type is None:
        return rho, u
    for k in range(1, len(wall_rho) + 1):
        sel = node_type == k
        rho[sel] = wall_rho[k - 1]
        for i in range(u.shape[0]):
            u[i][sel] = wall_u[k - 1][i]
    return rho, u


def random_case(lattice, dims, periodic, seed=0, u_amp=0.05, rho_amp=0.01, walls="none",
                n_wall_ids=2, force=None):
    """Random smooth-ish state; walls = 'none' | 'box' | 'mixed'.

    'box' closes every non-periodic axis with an outer layer of wall nodes;
    'mixed' also sprinkles interior obstacle nodes.  Wall ids cycle 1..n.
    """
    g = rng(seed)
    d = 2 if lattice == D2Q9 else 3
    grid = tuple(reversed(dims))
    rho = 1.0 + rho_amp * g.uniform(-1, 1, size=grid)
    u = u_amp * g.uniform(-1, 1, size=(d,) + grid)
    node_type = None
    wall_rho = wall_u = None
    if walls != "none":
        node_type = np.zeros(grid, dtype=np.uint8)
        for i in range(d):
            if not (periodic >> i) & 1:
                ax = d - 1 - i
                sl_lo = [slice(None)] * d
                sl_hi = [slice(None)] * d
                sl_lo[ax] = 0
                sl_hi[ax] = grid[ax] - 1
                node_type[tuple(sl_lo)] = 1 + (i % n_wall_ids)
                node_type[tuple(sl_hi)] = 1 + ((i + 1) % n_wall_ids)
        if walls == "mixed":
            interior = g.uniform(size=grid) < 0.05
            ids = g.integers(1, n_wall_ids + 1, size=grid).astype(np.uint8)
            node_type = np.where(interior & (node_type == 0), ids, node_type).astype(np.uint8)
        wall_rho = 1.0 + rho_amp * g.uniform(-1, 1, size=n_wall_ids)
        wall_u = u_amp * g.uniform(-1, 1, size=(n_wall_ids, d))
        rho, u = place_walls(rho, u, node_type, wall_rho, wall_u)
    return Case(lattice, tuple(dims), periodic, rho, u, node_type, wall_rho, wall_u,
                force=force, name=f"random-{walls}")


def tgv2d(n=64, u0=0.02):
    """Test 4 initial field on an n x n periodic D2Q9 grid, k = 2 pi / n.

    ux = -u0 cos(kx) sin(ky), uy = u0 sin(kx) cos(ky), rho = 1, at nodes 0..n-1.
    """
    k = 2.0 * math.pi / n
    x = np.arange(n) * k
    X, Y = np.meshgrid(x, x, indexing="xy")       # arrays are [y, x]
    u = np.stack([-u0 * np.cos(X) * np.sin(Y), u0 * np.sin(X) * np.cos(Y)])
    return Case(D2Q9, (n, n), 0b11, np.ones((n, n)), u, name=f"tgv2d-{n}")


def tgv3d(n=96, u0=0.02, noise_sigma=0.0, seed=5):
    """Standard 3D Taylor-Green field on an n^3 periodic D3Q19 grid.

    u = u0 sin kx cos ky cos kz, v = -u0 cos kx sin ky cos kz, w = 0, plus an
    optional seeded Gaussian perturbation of standard deviation noise_sigma.
    """
    k = 2.0 * math.pi / n
    x = np.arange(n) * k
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")  # arrays are [z, y, x]
    u = np.stack([u0 * np.sin(X) * np.cos(Y) * np.cos(Z),
                  -u0 * np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)])
    if noise_sigma > 0:
        u = u + noise_sigma * rng(seed).standard_normal(u.shape)
    return Case(D3Q19, (n, n, n), 0b111, np.ones((n, n, n)), u, name=f"tgv3d-{n}")


def lid_speed(re: float, n: int) -> float:
    """Lattice lid speed for a cavity of n nodes per side at Reynolds number re.

    At tau = 1 the lattice viscosity is 1/6, so Re = 6 U (n - 1) for a lid speed
    U (lattice units) over the n - 1 lattice spacings between the walls.
    """
    return re / (6.0 * (n - 1))


def cavity2d(n=256, lid=0.1, nx=None):
    """Test 3 set-up: closed D2Q9 box; walls id 1 (no-slip), lid id 2 on y = ny - 1.

    The lid holds the top-row nodes strictly between the side walls; the two
    top corners belong to the no-slip walls.
    """
    nx = nx or n
    ny = n
    nt = np.zeros((ny, nx), dtype=np.uint8)
    nt[0, :] = nt[-1, :] = 1
    nt[:, 0] = nt[:, -1] = 1
    nt[-1, 1:-1] = 2
    wall_rho = np.array([1.0, 1.0])
    wall_u = np.array([[0.0, 0.0], [lid, 0.0]])
    rho, u = place_walls(np.ones((ny, nx)), np.zeros((2, ny, nx)), nt, wall_rho, wall_u)
    return Case(D2Q9, (nx, ny), 0, rho, u, nt, wall_rho, wall_u, name=f"cavity2d-{nx}x{ny}")


def cavity3d(n=128, lid=0.1, nz=None):
    """Test 5 set-up: closed D3Q19 box (a cube unless nz is given); walls id 1,
    lid id 2 on z = nz - 1 moving +x.

    The lid holds the top-face nodes strictly inside the four side walls.
    """
    nz = nz or n
    nt = np.zeros((nz, n, n), dtype=np.uint8)
    nt[0], nt[-1] = 1, 1
    nt[:, 0, :], nt[:, -1, :] = 1, 1
    nt[:, :, 0], nt[:, :, -1] = 1, 1
    nt[-1, 1:-1, 1:-1] = 2
    wall_rho = np.array([1.0, 1.0])
    wall_u = np.array([[0.0, 0.0, 0.0], [lid, 0.0, 0.0]])
    rho, u = place_walls(np.ones((nz, n, n)), np.zeros((3, nz, n, n)), nt, wall_rho, wall_u)
    name = f"cavity3d-{n}" if nz == n else f"cavity3d-{n}x{n}x{nz}"
    return Case(D3Q19, (n, n, nz), 0, rho, u, nt, wall_rho, wall_u, name=name)


def channel2d(nx=20, ny=51, u_top=0.1, force_x=0.0):
    """Tests 1-2 set-up: periodic in x, plates at y = 0 (id 1, fixed) and y = ny - 1
    (id 2, moving at u_top).  force_x is the lattice-unit body-force increment."""
    nt = np.zeros((ny, nx), dtype=np.uint8)
    nt[0, :] = 1
    nt[-1, :] = 2
    wall_rho = np.array([1.0, 1.0])
    wall_u = np.array([[0.0, 0.0], [u_top, 0.0]])
    rho, u = place_walls(np.ones((ny, nx)), np.zeros((2, ny, nx)), nt, wall_rho, wall_u)
    return Case(D2Q9, (nx, ny), 0b01, rho, u, nt, wall_rho, wall_u,
                force=(force_x, 0.0), name=f"channel2d-{nx}x{ny}")


def batch_cavity_sides(count=64, seed=4):
    """Batched-cavity workload: sides uniform in {64, 96, ..., 512}, Re log-uniform
    in [100, 3200], lid speed from ``lid_speed`` capped at 1/6 (lattice units)."""
    g = rng(seed)
    sides = g.choice(np.arange(64, 513, 32), size=count)
    re = np.exp(g.uniform(math.log(100.0), math.log(3200.0), size=count))
    lids = np.minimum([lid_speed(r, int(s)) for r, s in zip(re, sides)], 1.0 / 6.0)
    return [int(s) for s in sides], [float(r) for r in re], [float(v) for v in lids]


def channel3d_sphere(nx=128, ny=128, nz=256, radius=None, force_z=1e-5, spin=0.0):
    """Obstacle workload: a D3Q19 channel along z (periodic in z) with no-slip
    side walls (id 1) at x = 0, nx - 1 and y = 0, ny - 1, and a sphere of nodes
    (id 2) centred in the channel a quarter of the way along z, driven by a
    body-force increment force_z along z (lattice units).

    spin != 0 gives the sphere a per-node wall velocity: rotation about the
    channel axis at angular rate spin (lattice units per lattice spacing), i.e.
    u = spin * (-(y - yc), x - xc, 0) on its nodes.  Returns (case, wall_u_field):
    wall_u_field is None without spin, else a [3, nz, ny, nx] velocity field
    that is nonzero only on the sphere's nodes (for per-node wall values).
    """
    radius = radius if radius is not None else min(nx, ny) / 8.0
    xc, yc, zc = (nx - 1) / 2.0, (ny - 1) / 2.0, nz / 4.0
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    nt = np.zeros((nz, ny, nx), dtype=np.uint8)
    nt[:, 0, :] = nt[:, -1, :] = 1
    nt[:, :, 0] = nt[:, :, -1] = 1
    sphere = (x - xc) ** 2 + (y - yc) ** 2 + (z - zc) ** 2 <= radius * radius
    nt[sphere & (nt == 0)] = 2
    wall_rho = np.array([1.0, 1.0])
    wall_u = np.zeros((2, 3))
    rho, u = place_walls(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)), nt, wall_rho, wall_u)
    field = None
    if spin != 0.0:
        field = np.zeros((3, nz, ny, nx))
        on = nt == 2
        field[0][on] = -spin * (y[on] - yc)
        field[1][on] = spin * (x[on] - xc)
        u = np.where(on[None], field, u)
    case = Case(D3Q19, (nx, ny, nz), 0b100, rho, u, nt, wall_rho, wall_u,
                force=(0.0, 0.0, force_z), name=f"channel3d-sphere-{nx}x{ny}x{nz}")
    return case, field
