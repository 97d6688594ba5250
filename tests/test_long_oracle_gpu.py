"""Long runs of the workload set against the FP64 CPU oracle itself.

The oracle runs its node loops on every host core (results bitwise equal to
one thread, tests/test_oracle_threads.py), which makes these full-size runs
affordable:

* the 2D lid-driven cavity, 256^2 nodes, Re 100 and 1000 (lid speed by
  Re = 6 U (N - 1), 0.065 and 0.65 lattice units), 20,000 steps: FP64 and FP32
  storage against the oracle;
* the 3D lid-driven cavity, 128^3 nodes, Re 100 and 400, 200 steps: FP64,
  FP32, BF16 and FP16 storage (FP32 arithmetic) against the oracle;
* the differentiable 96^3 Taylor-Green workload (u0 = 0.02 e plus a seeded
  perturbation, 2,000 steps): the gradient dL/du0 of the GPU rollout (FP32
  and FP64, sqrt(N)-checkpointed reverse pass) against the oracle's own
  reverse pass (chain rule of Eqs. (2), (4), (5), checkpointed), element by
  element.

Stated errors (relative L2 on u; measured on a GB300 with a 16-core host,
bars with a margin): 2D FP64 3e-13, FP32 2.6e-7 (Re 100) and 2.4e-4 (Re 1000:
the lid moves at 0.65 lattice units and FP32 rounding keeps the flow from
settling); 3D FP64 6e-14, FP32 1.3-2.4e-7, BF16 2-2.7e-2, FP16 5-7e-4.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()
    n = orc.set_threads(orc.host_cores())
    yield
    orc.set_threads(n)


def rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)))


def _gpu(case, precision, steps):
    s = M.Solver.from_case(case, precision)
    s.step(steps)
    r, u = s.get_state()
    s.close()
    return r, u


@pytest.mark.parametrize("re,tol32", [(100.0, 1e-6), (1000.0, 1e-3)])
def test_cavity2d_256_20k_steps_against_oracle(re, tol32):
    case = inputs.cavity2d(256, lid=inputs.lid_speed(re, 256))
    r_o, u_o = orc.step(case.lattice, case.rho, case.u, case.periodic, wall=case.wall_mask,
                        nsteps=20000)
    r64, u64 = _gpu(case, M.F64, 20000)
    r32, u32 = _gpu(case, M.F32, 20000)
    e64, e32 = rel_l2(u64, u_o), rel_l2(u32, u_o)
    print(f"256^2 Re {re:g}, 20k steps: FP64 {e64:.2e}, FP32 {e32:.2e}")
    assert e64 <= 1e-11
    assert np.abs(r64 - r_o).max() <= 1e-11
    assert e32 <= tol32


@pytest.mark.parametrize("re", [100.0, 400.0])
def test_cavity3d_128_200_steps_against_oracle(re):
    case = inputs.cavity3d(128, lid=inputs.lid_speed(re, 128))
    r_o, u_o = orc.step(case.lattice, case.rho, case.u, case.periodic, wall=case.wall_mask,
                        nsteps=200)
    bars = {M.F64: 1e-12, M.F32: 1e-6, M.F16_STORE: 3e-3, M.BF16_STORE: 8e-2}
    errs = {}
    for precision, tol in bars.items():
        r, u = _gpu(case, precision, 200)
        errs[precision] = rel_l2(u, u_o)
        assert errs[precision] <= tol, (precision, errs[precision])
    print(f"128^3 Re {re:g}, 200 steps:", {k: f"{v:.2e}" for k, v in errs.items()})


@pytest.fixture(scope="module")
def tgv96():
    """The differentiable workload and the oracle's gradient dL/du0 for
    L = ||u(T) - u_target||^2, u_target the analytic decayed field (dx = 1,
    nu = 1/6: e = 1, lattice and physical units coincide)."""
    n, steps, nu = 96, 2000, 1.0 / 6.0
    k = 2.0 * np.pi / n
    clean = inputs.tgv3d(n, 0.02)
    case = inputs.tgv3d(n, 0.02, noise_sigma=1e-3, seed=61)
    target = clean.u * np.exp(-3.0 * nu * k * k * steps)
    _, g_u0, _ = orc.rollout_adjoint(case.lattice, case.rho, case.u, 0b111, steps,
                                     lambda r, u: (np.zeros_like(r), 2.0 * (u - target)), None,
                                     checkpoint_every=45, gather=True)
    return case, target, steps, g_u0


@pytest.mark.parametrize("precision,tol", [(M.F32, 1e-4), (M.F64, 1e-10)])
def test_tgv3d_96_gradient_against_oracle_reverse_pass(tgv96, precision, tol):
    torch = pytest.importorskip("torch")
    from paper_1901_02716_gb300.adjoint import RolloutSpec, rollout
    case, target, steps, g_ref = tgv96
    spec = RolloutSpec(inputs.D3Q19, case.dims, 1.0, steps, 0b111, precision=precision)
    dt = torch.float64
    rho0 = torch.tensor(case.rho, dtype=dt, device="cuda")
    u0 = torch.tensor(case.u, dtype=dt, device="cuda", requires_grad=True)
    _, u_T = rollout(rho0, u0, None, 1.0 / 6.0, spec)
    loss = ((u_T - torch.tensor(target, dtype=dt, device="cuda")) ** 2).sum()
    loss.backward()
    g = u0.grad.cpu().numpy()
    v = inputs.rng(62).standard_normal(case.u.shape)
    err, err_v = rel_l2(g, g_ref), abs(float(np.sum(g * v)) / float(np.sum(g_ref * v)) - 1)
    print(f"96^3 TGV dL/du0 precision {precision}: rel L2 {err:.2e}, along v {err_v:.2e}")
    assert err <= tol and err_v <= tol
