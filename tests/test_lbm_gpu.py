"""The stream-and-collide comparator (maclab_lbm_*, the SRT-BGK LBM of Eq. (1)
that MacLAB replaces) against its FP64 oracle (oracle/lbm_tau1.py, pinned by an
exact rational BGK), and at tau = 1 against MacLAB itself on the GPU.

Bars: FP64 <= 1e-12 relative (max norm).  FP32 <= 4e-6 absolute on rho and
<= 5e-5 relative L2 on u after 40 steps: the stored distributions f ~ w rho
carry rho whole (no drho split), so each step rounds about 9 x 2^-24 x 0.4
into rho, a few times MacLAB's FP32 error (1e-6 on rho, 1e-5 on u with drho
storage)."""
import numpy as np
import pytest

from oracle import lbm_tau1
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu
D2 = inputs.D2Q9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


def rel_l2(a, b):
    return np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b))


@pytest.mark.parametrize("dims,tau", [((37, 23), 0.6), ((64, 48), 1.0), ((16, 65), 1.7), ((1, 9), 0.8)])
@pytest.mark.parametrize("precision", [M.F64, M.F32])
@pytest.mark.parametrize("steps", [1, 40])
def test_lbm_matches_oracle(dims, tau, precision, steps):
    case = inputs.random_case(D2, dims, 0b11, seed=51, u_amp=0.08, rho_amp=0.02)
    lb = M.Lbm(dims[0], dims[1], tau, precision)
    lb.set_state(case.rho, case.u)
    lb.step(steps)
    r_g, u_g = lb.get_state()
    assert lb.info()["steps"] == steps
    lb.close()
    r_o, u_o = lbm_tau1.run(case.rho, case.u, steps, tau=tau)
    if precision == M.F64:
        assert np.abs(r_g - r_o).max() <= 1e-12 * np.abs(r_o).max()
        assert np.abs(u_g - u_o).max() <= 1e-12 * np.abs(u_o).max()
    else:
        assert np.abs(r_g - r_o).max() <= 4e-6
        assert rel_l2(u_g, u_o) <= 5e-5


def test_lbm_at_tau_one_is_maclab():
    """Methods, Eqs. (9)-(13): at tau = 1 the stored-f scheme and MacLAB give
    the same (rho, u), here both on the GPU in FP64."""
    case = inputs.random_case(D2, (48, 40), 0b11, seed=52, u_amp=0.1, rho_amp=0.03)
    lb = M.Lbm(48, 40, 1.0, M.F64)
    lb.set_state(case.rho, case.u)
    lb.step(25)
    r_l, u_l = lb.get_state()
    lb.close()
    s = M.Solver.from_case(case, M.F64)
    e = s.params["e"]                      # physical u = e * lattice u (Eq. (6))
    s.step(25)
    r_m, u_m = s.get_state()
    s.close()
    assert np.abs(r_l - r_m).max() <= 1e-12
    assert np.abs(u_l - u_m / e).max() <= 1e-12 * np.abs(u_l).max()


def test_lbm_conserves_mass_and_momentum():
    case = inputs.random_case(D2, (96, 64), 0b11, seed=53, u_amp=0.08, rho_amp=0.03)
    lb = M.Lbm(96, 64, 0.7, M.F64)
    lb.set_state(case.rho, case.u)
    lb.step(100)
    r, u = lb.get_state()
    lb.close()
    assert abs(r.sum() - case.rho.sum()) <= 1e-11 * case.rho.sum()
    for i in range(2):
        assert abs((r * u[i]).sum() - (case.rho * case.u[i]).sum()) <= 1e-11 * case.rho.sum()


def test_lbm_rejects_bad_arguments():
    for args in ((0, 8, 1.0, M.F32), (8, 8, 0.5, M.F32), (8, 8, 1.0, M.BF16_STORE)):
        with pytest.raises(M.MacLABError) as ei:
            M.Lbm(*args)
        assert ei.value.status == M.ERR_INVALID


def test_lbm_state_footprint():
    lb = M.Lbm(1024, 1024, 0.8, M.F32)
    info = lb.info()
    lb.close()
    assert info["state_bytes"] == 2 * 9 * 1024 * 1024 * 4 and info["bytes_per_update"] == 72
