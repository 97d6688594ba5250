"""Slab decomposition on the GPU: k slabs of the CUDA library on one GPU,
ghost planes exchanged through device buffers (maclab_get_planes /
maclab_set_planes) after every step, against the undivided domain.

A radius-1 stencil sees the same upstream values in both, and the step kernels
sum each node's terms in the same order whatever the chunking of the march
axis, so the slabs' interiors equal the undivided GPU run bit for bit (FP32 and
FP64), and the oracle within the usual bars.  The diagnostics added over slabs
(maclab_diagnostics_sums) match the undivided domain's.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs, slabs
from paper_1901_02716_gb300 import maclab as M
from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


CASES = [
    ("tgv3d", lambda: inputs.tgv3d(32, 0.05, noise_sigma=1e-3, seed=9), 2, 12),
    ("tgv3d-3", lambda: inputs.tgv3d(32, 0.05, noise_sigma=1e-3, seed=9), 3, 12),
    ("cavity3d", lambda: inputs.cavity3d(32, lid=0.1), 2, 12),
    ("channel2d", lambda: inputs.channel2d(nx=32, ny=40, u_top=0.1, force_x=1e-4), 2, 20),
    ("sphere", lambda: inputs.channel3d_sphere(nx=32, ny=32, nz=48, radius=5.0, force_z=1e-4)[0], 2, 10),
]


@pytest.mark.parametrize("name,make,k,steps", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [M.F32, M.F64])
def test_slabs_equal_undivided_run(name, make, k, steps, precision):
    case = make()
    s = M.Solver.from_case(case, precision)
    s.step(steps)
    r1, u1 = s.get_state()
    d1 = s.diagnostics()
    s.close()
    dom = slabs.SlabDomain(case, k, precision)
    dom.step(steps)
    r2, u2 = dom.get_state()
    d2 = dom.diagnostics()
    dom.close()
    assert np.array_equal(r1, r2) and np.array_equal(u1, u2)
    assert d2["mass"] == pytest.approx(d1["mass"], rel=1e-12)
    assert d2["kinetic"] == pytest.approx(d1["kinetic"], rel=1e-12)
    assert d2["residual"] == pytest.approx(d1["residual"], rel=1e-10)
    # deeper halos: fewer exchanges, same interiors
    dom = slabs.SlabDomain(case, k, precision, depth=4)
    dom.step(steps)
    r3, u3 = dom.get_state()
    dom.close()
    assert np.array_equal(r1, r3) and np.array_equal(u1, u3)
    r_o, u_o = orc.step(case.lattice, case.rho, case.u, case.periodic, wall=case.wall_mask,
                        force=case.force, nsteps=steps)
    assert_parity(r2, u2, r_o, u_o, precision)
