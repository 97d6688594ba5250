"""Per-node wall values (maclab_set_wall_state) against the FP64 oracle.

The paper keeps the physical variables of wall nodes and computes nothing there
(boundary treatment of Tests 1-3 and 5); wall nodes still act as upstream
sources of their fluid neighbours.  The oracle implements exactly that for
whatever values its input holds on wall nodes, so per-node wall values are
checked by giving both sides the same field:

* random per-node wall fields on box walls and random obstacle masks, D2Q9 and
  D3Q19, FP64 and FP32 storage;
* wall values changed between steps (a time-dependent boundary);
* maclab_set_state afterwards puts the wall-id table's values back;
* the obstacle workload at full size: a 128 x 128 x 256 channel with no-slip
  side walls and a sphere spinning about the channel axis (per-node wall
  velocity), driven by a body force, 3 steps, element by element.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M
from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()
    n = orc.set_threads(orc.host_cores())
    yield
    orc.set_threads(n)


def _wall_field(case, seed):
    """Random physical (rho, u) on the wall nodes; garbage elsewhere (not read)."""
    g = inputs.rng(seed)
    rho = 1.0 + 0.02 * g.uniform(-1, 1, size=case.grid)
    u = 0.08 * g.uniform(-1, 1, size=(case.d,) + case.grid)
    return rho, u


def _with_walls(case, rho_w, u_w):
    w = case.wall_mask
    rho = np.where(w, rho_w, case.rho)
    u = np.where(w[None], u_w, case.u)
    return rho, u


CASES = [
    (inputs.D2Q9, (40, 24), 0b01, "box"),
    (inputs.D2Q9, (33, 20), 0b00, "mixed"),
    (inputs.D3Q19, (32, 16, 12), 0b000, "box"),
    (inputs.D3Q19, (64, 24, 13), 0b110, "mixed"),
    (inputs.D3Q19, (20, 16, 17), 0b100, "mixed"),
]


@pytest.mark.parametrize("lat,dims,periodic,walls", CASES)
@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_per_node_wall_values(lat, dims, periodic, walls, precision):
    case = inputs.random_case(lat, dims, periodic, seed=71, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=tuple([1e-4] * len(dims)))
    rho_w, u_w = _wall_field(case, 72)
    s = M.Solver.from_case(case, precision)
    s.set_wall_state(rho_w, u_w)
    s.step(6)
    r_g, u_g = s.get_state()
    s.close()
    rho0, u0 = _with_walls(case, rho_w, u_w)
    r_o, u_o = orc.step(lat, rho0, u0, periodic, wall=case.wall_mask, force=case.force, nsteps=6)
    assert_parity(r_g, u_g, r_o, u_o, precision)
    # the wall nodes kept the given values
    w = case.wall_mask
    tol = 1e-15 if precision == M.F64 else 1e-7
    assert np.abs(u_g[:, w] - u_w[:, w]).max() <= tol
    assert np.abs(r_g[w] - rho_w[w]).max() <= tol


@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_wall_values_changed_between_steps(precision):
    case = inputs.random_case(inputs.D3Q19, (32, 16, 12), 0b100, seed=73, u_amp=0.08, rho_amp=0.02,
                              walls="mixed")
    f1, f2 = _wall_field(case, 74), _wall_field(case, 75)
    s = M.Solver.from_case(case, precision)
    s.set_wall_state(*f1)
    s.step(3)
    s.set_wall_state(*f2)
    s.step(4)
    r_g, u_g = s.get_state()
    s.close()
    r_o, u_o = orc.step(case.lattice, *_with_walls(case, *f1), case.periodic, wall=case.wall_mask,
                        nsteps=3)
    mid = inputs.Case(case.lattice, case.dims, case.periodic, r_o, u_o, case.node_type)
    r_o, u_o = orc.step(case.lattice, *_with_walls(mid, *f2), case.periodic, wall=case.wall_mask,
                        nsteps=4)
    assert_parity(r_g, u_g, r_o, u_o, precision)


def test_set_state_restores_table_values():
    case = inputs.random_case(inputs.D2Q9, (40, 24), 0b01, seed=76, walls="box")
    s = M.Solver.from_case(case, M.F64)
    s.set_wall_state(*_wall_field(case, 77))
    s.set_state(case.rho, case.u)
    r, u = s.get_state()
    s.close()
    w = case.wall_mask
    assert np.array_equal(r[w], case.rho[w]) and np.array_equal(u[:, w], case.u[:, w])


@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_spinning_sphere_channel_full_size(precision):
    """The obstacle workload at full size: 128 x 128 x 256, mask mode."""
    case, field = inputs.channel3d_sphere(spin=0.01)
    s = M.Solver.from_case(case, precision)
    rho_w = np.ones(case.grid)
    s.set_wall_state(rho_w, field)
    s.step(3)
    r_g, u_g = s.get_state()
    s.close()
    u0 = np.where(case.wall_mask[None], field, case.u)
    r_o, u_o = orc.step(case.lattice, case.rho, u0, case.periodic, wall=case.wall_mask,
                        force=case.force, nsteps=3)
    assert_parity(r_g, u_g, r_o, u_o, precision)
