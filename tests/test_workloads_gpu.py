"""The long runs of the workload set on the GPU, with the error of every
storage type stated against the FP64 path (itself held to the FP64 oracle at
1e-12 per step by test_parity_gpu.py; the CPU oracle would need hours for
these step counts):

* 2D lid-driven cavities, 256^2 and 1024^2, Re 100 and 1000, 20,000 steps:
  FP32 (drho storage) against FP64, and the FP64 steady residual;
* the 3D lid-driven cavity, 128^3, Re 100 and 400, 10,000 steps: FP32, BF16
  and FP16 storage (FP32 arithmetic) against FP64.

The bounds are the stated errors (measured values in the results, with a
margin): FP32 stays within 1e-5 relative L2 on u except the 256^2, Re 1000
cavity, whose lid moves at 0.65 lattice units (Re = 6 U (N - 1) at tau = 1)
and where FP32 rounding keeps the flow from settling (2.4e-4); 16-bit storage
accumulates its rounding over 10,000 steps (BF16 11-26 %, FP16 1.5-3 %).
About 30 s of GPU time."""
import numpy as np
import pytest

from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


def rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)))


def _run(case, precision, steps):
    s = M.Solver.from_case(case, precision)
    s.step(steps)
    d = s.diagnostics()
    r, u = s.get_state()
    s.close()
    return r, u, d


@pytest.mark.parametrize("n,re,u_tol", [(256, 100.0, 1e-5), (256, 1000.0, 1e-3), (1024, 100.0, 1e-5),
                                        (1024, 1000.0, 1e-5)])
def test_cavity2d_20k_steps_fp32_vs_fp64(n, re, u_tol):
    case = inputs.cavity2d(n, lid=inputs.lid_speed(re, n))
    r64, u64, d64 = _run(case, M.F64, 20000)
    r32, u32, d32 = _run(case, M.F32, 20000)
    assert np.isfinite(u32).all() and np.isfinite(u64).all()
    assert rel_l2(u32, u64) <= u_tol
    assert 0.0 < d64["residual"] < 1e-4             # FP64 steady residual ||u^n - u^n-1|| / ||u^n||
    assert d64["nonfinite"] == 0 and d32["nonfinite"] == 0


@pytest.mark.parametrize("re", [100.0, 400.0])
def test_cavity3d_10k_steps_storage_errors(re):
    case = inputs.cavity3d(128, lid=inputs.lid_speed(re, 128))
    r64, u64, d64 = _run(case, M.F64, 10000)
    assert 0.0 < d64["residual"] < 1e-5
    bounds = {M.F32: 5e-6, M.F16_STORE: 6e-2, M.BF16_STORE: 5e-1}
    for precision, tol in bounds.items():
        r, u, d = _run(case, precision, 10000)
        assert d["nonfinite"] == 0
        assert rel_l2(u, u64) <= tol, (precision, rel_l2(u, u64))
