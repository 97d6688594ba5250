"""GPU diagnostics (FP64 reductions), CUDA-graph stepping and fault reporting.

Diagnostics are checked against plain FP64 sums of the oracle's fields; the
non-finite check is exercised by planting a NaN in the host input (the fault
is made on the host, never on the GPU).
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu
D2, D3 = inputs.D2Q9, inputs.D3Q19


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


@pytest.mark.parametrize("lat,dims,periodic,walls", [
    (D2, (40, 23), 0b01, "mixed"), (D2, (64, 48), 0b11, "none"),
    (D3, (16, 12, 10), 0b000, "box"), (D3, (12, 9, 8), 0b101, "mixed")])
@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_diagnostics_match_oracle_sums(lat, dims, periodic, walls, precision):
    case = inputs.random_case(lat, dims, periodic, seed=51, u_amp=0.08, rho_amp=0.02, walls=walls)
    s = M.Solver.from_case(case, precision)
    s.step(3)
    d = s.diagnostics()
    r_o, u_o = orc.step(lat, case.rho, case.u, periodic, wall=case.wall_mask, nsteps=3)
    r_p, u_p = orc.step(lat, case.rho, case.u, periodic, wall=case.wall_mask, nsteps=2)
    fluid = None if case.node_type is None else case.node_type == 0
    ref = orc.diagnostics(r_o, u_o, u_prev=u_p, fluid=fluid)
    tol = 1e-12 if precision == M.F64 else 1e-6
    assert d["mass"] == pytest.approx(ref["mass"], rel=tol)
    assert d["kinetic"] == pytest.approx(ref["kinetic"], rel=max(tol, 1e-12) * 10)
    for i in range(len(dims)):
        assert abs(d["momentum"][i] - ref["momentum"][i]) < 10 * tol * ref["mass"] * 0.1
    assert d["residual"] == pytest.approx(ref["residual"], rel=1e-9 if precision == M.F64 else 1e-3)
    umax = np.sqrt(np.sum(u_o ** 2, axis=0))
    if fluid is not None:
        umax = umax[fluid]
    assert d["max_u_lattice"] == pytest.approx(umax.max(), rel=1e-12 if precision == M.F64 else 1e-6)
    assert d["nonfinite"] == 0
    s.close()


def test_residual_unavailable_after_set_state():
    case = inputs.random_case(D2, (32, 16), 0b11, seed=52)
    s = M.Solver.from_case(case, M.F32)
    assert s.diagnostics()["residual"] == -1
    s.step(1)
    assert s.diagnostics()["residual"] > 0
    s.close()


def test_fp32_conservation_on_periodic_grid():
    """Eq. (15): mass and momentum are invariants; FP32 storage with FP64 sums
    keeps the drift at the level of FP32 rounding."""
    case = inputs.tgv3d(32, 0.05)
    s = M.Solver.from_case(case, M.F32)
    d0 = s.diagnostics()
    s.step(1000)
    d1 = s.diagnostics()
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-6)
    for i in range(3):
        assert abs(d1["momentum"][i] - d0["momentum"][i]) < 1e-6 * d0["mass"]
    s.close()


def test_nonfinite_is_reported():
    case = inputs.random_case(D2, (32, 16), 0b11, seed=53)
    rho = case.rho.copy()
    rho[3, 5] = np.nan            # planted on the host
    s = M.Solver(D2, case.dims, 1.0, 1 / 6, M.F32, case.periodic)
    s.set_state(rho, case.u.copy())
    with pytest.raises(M.MacLABError) as ei:
        s.diagnostics()
    assert ei.value.status == M.ERR_NONFINITE
    d = s.diagnostics(raise_nonfinite=False)
    assert d["nonfinite"] == 1
    s.step(2)                     # the NaN spreads to the 9 nodes downstream of it, then 25
    assert s.diagnostics(raise_nonfinite=False)["nonfinite"] == 25
    s.close()


@pytest.mark.parametrize("lat,dims,periodic,walls", [(D2, (64, 40), 0b00, "box"),
                                                     (D3, (32, 16, 12), 0b011, "box")])
def test_graph_stepping_is_bit_identical(lat, dims, periodic, walls):
    case = inputs.random_case(lat, dims, periodic, seed=54, walls=walls)
    out = []
    for g in (0, 8, 6):
        s = M.Solver.from_case(case, M.F32)
        s.set_graph(g)
        s.step(37)
        out.append(s.get_lattice_state().copy())
        assert s.params["steps"] == 37
        s.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


@pytest.mark.parametrize("lat,dims,periodic,walls", [
    (D2, (40, 23), 0b01, "mixed"), (D3, (16, 12, 10), 0b000, "box")])
def test_device_sums_equal_host_sums(lat, dims, periodic, walls):
    """maclab_diagnostics_device leaves in device memory the same raw sums,
    bit for bit, that maclab_diagnostics_sums returns to the host."""
    import torch
    case = inputs.random_case(lat, dims, periodic, seed=53, u_amp=0.08, rho_amp=0.02, walls=walls)
    s = M.Solver.from_case(case, M.F32)
    s.step(2)
    host = np.asarray(M.maclab_diagnostics_sums(s.handle))
    out = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    M.maclab_diagnostics_device(s.handle, out)
    s.sync()
    assert np.array_equal(out.cpu().numpy(), host)
    s.close()
