"""GPU adjoint against the FP64 oracle adjoint and central finite differences.

* one reverse step (maclab_adjoint_step) against oracle.adjoint_step;
* a whole differentiable rollout (torch.autograd) against the oracle's
  reverse pass for the initial field, and against central differences of the
  FP64 oracle forward for the wall velocity and nu;
* sqrt(N) checkpointing gives exactly the gradient of storing every state.
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


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


def _raw(torch, s):
    buf = torch.empty(s.state_bytes(), dtype=torch.uint8, device="cuda")
    s.get_lattice_state(buf)
    return buf


@pytest.mark.parametrize("lat,dims,periodic,walls", [
    (D2, (24, 17), 0b11, "none"), (D2, (20, 15), 0b01, "mixed"), (D2, (17, 13), 0b00, "box"),
    (D3, (8, 8, 6), 0b111, "none"), (D3, (12, 9, 8), 0b000, "box"), (D3, (9, 8, 7), 0b101, "mixed")])
@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_adjoint_step_matches_oracle(torch, lat, dims, periodic, walls, precision):
    d = len(dims)
    case = inputs.random_case(lat, dims, periodic, seed=71, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=tuple([3e-4] * d))
    s = M.Solver.from_case(case, precision)        # e = 1, rho0 = 1: physical == lattice
    s0 = _raw(torch, s)
    s.step(1)
    s1 = _raw(torch, s)
    g = inputs.rng(72)
    lr1 = g.standard_normal(case.rho.shape)
    lu1 = g.standard_normal(case.u.shape)
    dt = torch.float64
    lam1 = torch.empty(s.adjoint_bytes(), dtype=torch.uint8, device="cuda")
    lam0 = torch.empty_like(lam1)
    M.maclab_adjoint_seed(s.handle, torch.tensor(lr1, dtype=dt, device="cuda"),
                          torch.tensor(lu1, dtype=dt, device="cuda"), s1, lam1)
    gf = torch.zeros(3, dtype=torch.float64, device="cuda")
    M.maclab_adjoint_step(s.handle, s0, s1, lam1, lam0, gf)
    gr = torch.empty(case.rho.shape, dtype=dt, device="cuda")
    gu = torch.empty(case.u.shape, dtype=dt, device="cuda")
    nw = 0 if case.wall_u is None else len(case.wall_u)
    res = M.maclab_adjoint_finish(s.handle, lam0, s0, gr, gu, 0.0, gf.cpu().tolist(), nw)
    s.close()
    lr0, lu0, gfo = orc.adjoint_step(lat, case.rho, case.u, periodic, lr1, lu1,
                                     wall=case.wall_mask, force=case.force)
    tol = 1e-11 if precision == M.F64 else 2e-5
    fluid = np.ones(case.rho.shape, bool) if case.node_type is None else case.node_type == 0
    scale_r = np.abs(lr0).max()
    scale_u = np.abs(lu0).max()
    assert np.abs(gr.cpu().numpy()[fluid] - lr0[fluid]).max() <= tol * scale_r
    assert np.abs(gu.cpu().numpy()[:, fluid] - lu0[:, fluid]).max() <= tol * scale_u
    # sum of lam_u' over fluid nodes; in FP32 the adjoint array rounds lam_u' to float
    gtol = 1e-12 if precision == M.F64 else 1e-6
    assert np.abs(gf.cpu().numpy()[:d] - gfo).max() <= gtol * np.abs(gfo).max() * np.sqrt(lu1.size)
    for k in range(nw):
        sel = case.node_type == k + 1
        assert res["wall"][k][0] == pytest.approx(lr0[sel].sum(), rel=tol * 10, abs=tol * scale_r)
        for i in range(d):
            assert res["wall"][k][1 + i] == pytest.approx(lu0[i][sel].sum(), rel=tol * 10,
                                                          abs=tol * scale_u)


@pytest.mark.parametrize("lat,dims,periodic,walls", [
    (D2, (24, 17), 0b11, "none"), (D2, (20, 15), 0b01, "mixed"), (D2, (17, 13), 0b00, "box"),
    (D3, (8, 8, 6), 0b111, "none"), (D3, (12, 9, 8), 0b000, "box"), (D3, (9, 8, 7), 0b101, "mixed"),
    # shapes of the two-rows kernel's viscosity mode (FP32): rows of 2 to 32 quads,
    # idle lanes, obstacle masks, box walls, every periodicity
    (D3, (16, 8, 7), 0b101, "mixed"), (D3, (32, 16, 9), 0b000, "box"), (D3, (128, 8, 6), 0b010, "box"),
    (D3, (4, 16, 5), 0b000, "box"), (D3, (40, 8, 12), 0b111, "none")])
@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_viscosity_term_matches_oracle(torch, lat, dims, periodic, walls, precision):
    """maclab_adjoint_nu_term (one reverse step's share of e dL/de) against the
    oracle's plain definition (pinned on the CPU by finite differences in e):
    the per-node kernel (no state after the step given) and, given that state,
    the tiled pass where it is built."""
    d = len(dims)
    case = inputs.random_case(lat, dims, periodic, seed=74, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=tuple([3e-4] * d))
    s = M.Solver.from_case(case, precision)        # e = 1, rho0 = 1: physical == lattice
    s0 = _raw(torch, s)
    g = inputs.rng(75)
    lr1 = g.standard_normal(case.rho.shape)
    lu1 = g.standard_normal(case.u.shape)
    dt = torch.float64
    lam1 = torch.empty(s.adjoint_bytes(), dtype=torch.uint8, device="cuda")
    s.step(1)
    s1 = _raw(torch, s)
    M.maclab_adjoint_seed(s.handle, torch.tensor(lr1, dtype=dt, device="cuda"),
                          torch.tensor(lu1, dtype=dt, device="cuda"), s1, lam1)
    acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    acc_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    M.maclab_adjoint_nu_term(s.handle, s0, lam1, acc)
    M.maclab_adjoint_nu_term(s.handle, s0, lam1, acc_t, s1)
    got, got_t = float(acc.item()), float(acc_t.item())
    s.close()
    ref = orc.nu_term(lat, case.rho, case.u, periodic, lr1, lu1, wall=case.wall_mask, force=case.force)
    tol = 1e-10 if precision == M.F64 else 1e-4
    assert got == pytest.approx(ref, rel=tol)
    assert got_t == pytest.approx(ref, rel=tol)


def _cavity_problem(n=20, lid=0.08, dx=0.05, nu=0.02, precision=M.F64, steps=25, seg=0):
    from paper_1901_02716_gb300.adjoint import RolloutSpec
    case = inputs.cavity2d(n, lid=lid)
    e, _ = orc.params(dx, nu)
    spec = RolloutSpec(D2, case.dims, dx, steps, case.periodic, case.node_type, case.wall_rho,
                       precision, checkpoint_every=seg)
    g = inputs.rng(73)
    u0 = 0.01 * e * g.standard_normal(case.u.shape)
    rho0 = 1.0 + 0.01 * g.standard_normal(case.rho.shape)
    target = 0.02 * e * g.standard_normal(case.u.shape)
    wall_u = np.asarray(case.wall_u) * e          # physical, [2, 2]
    return case, spec, rho0, u0, wall_u, target, e


def _oracle_loss(case, dx, nu, rho0, u0, wall_u, target, steps):
    e, _ = orc.params(dx, nu)
    rl, ul = inputs.place_walls(rho0, u0 / e, case.node_type, case.wall_rho, wall_u / e)
    r, u = orc.step(D2, rl, ul, case.periodic, wall=case.wall_mask, nsteps=steps)
    return float(np.sum((u * e - target) ** 2))


@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_rollout_without_viscosity_gradient(torch, precision):
    """With nu not differentiated the reverse pass skips the viscosity term:
    no gradient for nu, and the other gradients those of a rollout that also
    differentiates nu (the term only reads the adjoint): the initial field's
    bit for bit, the wall ids' to 1e-12 (their sums over wall nodes are FP64
    atomics, whose order varies from run to run)."""
    from paper_1901_02716_gb300.adjoint import rollout
    dx, nu, steps = 0.05, 0.02, 12
    case, spec, rho0, u0, wall_u, target, e = _cavity_problem(dx=dx, nu=nu, precision=precision,
                                                             steps=steps, seg=5)
    dt = torch.float64
    grads = []
    for nu_grad in (True, False):
        u0_t = torch.tensor(u0, dtype=dt, device="cuda", requires_grad=True)
        wall_t = torch.tensor(wall_u, dtype=dt, device="cuda", requires_grad=True)
        nu_t = torch.tensor(nu, dtype=dt, requires_grad=nu_grad)
        r_T, u_T = rollout(torch.tensor(rho0, dtype=dt, device="cuda"), u0_t, wall_t, nu_t, spec)
        ((u_T - torch.tensor(target, dtype=dt, device="cuda")) ** 2).sum().backward()
        grads.append((u0_t.grad.clone(), wall_t.grad.clone(), nu_t.grad))
    assert grads[0][2] is not None and grads[1][2] is None
    assert torch.equal(grads[0][0], grads[1][0])
    assert torch.allclose(grads[0][1], grads[1][1], rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("precision,tol", [(M.F64, 1e-7), (M.F32, 1e-4)])
def test_rollout_gradients(torch, precision, tol):
    from paper_1901_02716_gb300.adjoint import rollout
    dx, nu, steps = 0.05, 0.02, 25
    case, spec, rho0, u0, wall_u, target, e = _cavity_problem(dx=dx, nu=nu, precision=precision,
                                                             steps=steps)
    dt = torch.float64
    rho0_t = torch.tensor(rho0, dtype=dt, device="cuda", requires_grad=True)
    u0_t = torch.tensor(u0, dtype=dt, device="cuda", requires_grad=True)
    wall_t = torch.tensor(wall_u, dtype=dt, device="cuda", requires_grad=True)
    nu_t = torch.tensor(nu, dtype=dt, requires_grad=True)
    target_t = torch.tensor(target, dtype=dt, device="cuda")
    r_T, u_T = rollout(rho0_t, u0_t, wall_t, nu_t, spec)
    loss = ((u_T - target_t) ** 2).sum()
    loss.backward()
    # forward value against the oracle
    ref = _oracle_loss(case, dx, nu, rho0, u0, wall_u, target, steps)
    assert float(loss) == pytest.approx(ref, rel=1e-10 if precision == M.F64 else 1e-5)
    # initial-field gradient against the oracle reverse pass (lattice -> physical)
    rl, ul = inputs.place_walls(rho0, u0 / e, case.node_type, case.wall_rho, wall_u / e)
    r, u = orc.step(D2, rl, ul, case.periodic, wall=case.wall_mask, nsteps=steps)
    lam_u_T = 2 * (u * e - target) * e
    lr0, lu0, _ = orc.rollout_adjoint(D2, rl, ul, case.periodic, steps, np.zeros_like(r), lam_u_T,
                                      wall=case.wall_mask)
    fluid = case.node_type == 0
    gu_ref = np.where(fluid, lu0 / e, 0.0)
    gu = u0_t.grad.cpu().numpy()
    assert np.abs(gu - gu_ref).max() <= tol * np.abs(gu_ref).max()
    gr_ref = np.where(fluid, lr0, 0.0)
    assert np.abs(rho0_t.grad.cpu().numpy() - gr_ref).max() <= tol * np.abs(gr_ref).max()
    # wall velocity and viscosity against central differences of the FP64 oracle
    # (4-point stencil, step 1e-3 relative: truncation and round-off ~1e-11)
    def wall_loss(dw):
        w = wall_u.copy()
        w[1, 0] += dw
        return _oracle_loss(case, dx, nu, rho0, u0, w, target, steps)
    fd_w = fd4(wall_loss, 1e-3 * e)
    assert wall_t.grad[1, 0].item() == pytest.approx(fd_w, rel=tol)
    fd_nu = fd4(lambda d: _oracle_loss(case, dx, nu + d, rho0, u0, wall_u, target, steps), 1e-3 * nu)
    assert nu_t.grad.item() == pytest.approx(fd_nu, rel=tol)


def fd4(f, h):
    """Fourth-order central difference of f at 0."""
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


def test_checkpointing_is_exact(torch):
    from paper_1901_02716_gb300.adjoint import rollout
    grads = []
    for seg in (1, 5, 0, 25):
        case, spec, rho0, u0, wall_u, target, e = _cavity_problem(precision=M.F32, seg=seg)
        u0_t = torch.tensor(u0, dtype=torch.float32, device="cuda", requires_grad=True)
        rho0_t = torch.tensor(rho0, dtype=torch.float32, device="cuda")
        wall_t = torch.tensor(wall_u, dtype=torch.float32, device="cuda", requires_grad=True)
        r_T, u_T = rollout(rho0_t, u0_t, wall_t, 0.02, spec)
        ((u_T - torch.tensor(target, dtype=torch.float32, device="cuda")) ** 2).sum().backward()
        grads.append((u0_t.grad.cpu().numpy(), wall_t.grad.cpu().numpy()))
    for g in grads[1:]:
        assert np.array_equal(g[0], grads[0][0])
        # per-wall sums are FP64 atomic additions: equal up to their order
        assert np.allclose(g[1], grads[0][1], rtol=1e-12, atol=0)


def test_body_force_gradient(torch):
    """Poiseuille channel: the gradient with respect to the body acceleration
    against central differences of the oracle."""
    dx, nu, steps = 0.02, 0.003, 30
    case = inputs.channel2d(20, 21, u_top=0.0)
    e, dt_phys = orc.params(dx, nu)
    accel = 1e-4
    s = M.Solver(D2, case.dims, dx, nu, M.F64, case.periodic, case.node_type, case.wall_rho,
                 np.asarray(case.wall_u) * e, body_force=(accel, 0.0))
    g = inputs.rng(74)
    u0 = 0.005 * e * g.standard_normal(case.u.shape)
    s.set_state(case.rho.copy(), u0)
    states = [_raw(torch, s)]
    for _ in range(steps):
        s.step(1)
        states.append(_raw(torch, s))
    r_T, u_T = s.get_state()
    w = inputs.rng(75).standard_normal(case.u.shape)
    lam = torch.empty(s.adjoint_bytes(), dtype=torch.uint8, device="cuda")
    lam2 = torch.empty_like(lam)
    dot = M.maclab_adjoint_seed(s.handle, None, torch.tensor(w, device="cuda"), states[-1], lam)
    gf = torch.zeros(3, dtype=torch.float64, device="cuda")
    for k in range(steps - 1, -1, -1):
        M.maclab_adjoint_step(s.handle, states[k], states[k + 1], lam, lam2, gf)
        lam, lam2 = lam2, lam
    gr = torch.empty(case.rho.shape, dtype=torch.float64, device="cuda")
    gu = torch.empty(case.u.shape, dtype=torch.float64, device="cuda")
    res = M.maclab_adjoint_finish(s.handle, lam, states[0], gr, gu, dot, gf.cpu().tolist(), 2)
    s.close()

    def loss(a):
        f = orc.force_lattice([a, 0.0], dx, nu)
        rl, ul = inputs.place_walls(case.rho, u0 / e, case.node_type, case.wall_rho, case.wall_u)
        r, u = orc.step(D2, rl, ul, case.periodic, wall=case.wall_mask, force=f, nsteps=steps)
        return float(np.sum(u * e * w))
    fd = fd4(lambda d: loss(accel + d), 1e-3 * accel)
    assert res["accel"][0] == pytest.approx(fd, rel=1e-7)


@pytest.mark.parametrize("lat,dims,periodic,walls", [
    (D2, (64, 37), 0b00, "box"), (D2, (96, 41), 0b01, "mixed"), (D2, (4, 9), 0b11, "none"),
    (D2, (1024, 6), 0b10, "box"),
    (D3, (32, 16, 7), 0b011, "box"), (D3, (20, 13, 17), 0b100, "mixed"), (D3, (8, 8, 5), 0b111, "none"),
    (D3, (128, 12, 6), 0b000, "box"), (D3, (256, 6, 5), 0b101, "mixed"), (D3, (64, 8, 9), 0b111, "none")])
@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_tiled_adjoint_matches_reference_adjoint(torch, lat, dims, periodic, walls, precision):
    """The tiled reverse step (pair records, staged pull gather) against the
    reference two-kernel reverse step, on the same stored states."""
    d = len(dims)
    case = inputs.random_case(lat, dims, periodic, seed=76, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=tuple([2e-4] * d))
    out = []
    for kern in (M.KERNEL_REFERENCE, M.KERNEL_AUTO):
        s = M.Solver.from_case(case, precision)
        s.set_kernel(kern)
        s0 = _raw(torch, s)
        s.step(1)
        s1 = _raw(torch, s)
        g = inputs.rng(77)
        dt = torch.float64
        lam1 = torch.empty(s.adjoint_bytes(), dtype=torch.uint8, device="cuda")
        lam0 = torch.empty_like(lam1)
        M.maclab_adjoint_seed(s.handle, torch.tensor(g.standard_normal(case.rho.shape), dtype=dt,
                                                     device="cuda"),
                              torch.tensor(g.standard_normal(case.u.shape), dtype=dt, device="cuda"),
                              s1, lam1)
        gf = torch.zeros(3, dtype=torch.float64, device="cuda")
        M.maclab_adjoint_step(s.handle, s0, s1, lam1, lam0, gf)
        gr = torch.empty(case.rho.shape, dtype=dt, device="cuda")
        gu = torch.empty(case.u.shape, dtype=dt, device="cuda")
        nw = 0 if case.wall_u is None else len(case.wall_u)
        res = M.maclab_adjoint_finish(s.handle, lam0, s0, gr, gu, 0.0, gf.cpu().tolist(), nw)
        out.append((gr.cpu().numpy(), gu.cpu().numpy(), res["wall"], gf.cpu().numpy()))
        s.close()
    (r1, u1, w1, f1), (r2, u2, w2, f2) = out
    tol = 1e-12 if precision == M.F64 else 2e-6
    assert np.abs(r1 - r2).max() <= tol * np.abs(r1).max()
    assert np.abs(u1 - u2).max() <= tol * np.abs(u1).max()
    assert np.allclose(w1, w2, rtol=tol * 10, atol=tol * max(np.abs(r1).max(), np.abs(u1).max()))
    assert np.allclose(f1, f2, rtol=1e-6 if precision == M.F32 else 1e-12)
