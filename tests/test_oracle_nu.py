"""Pin of the oracle's viscosity term (oracle.nu_term) on the CPU.

nu enters a rollout only through the particle speed e = 6 nu / dx of Eq. (6):
the lattice velocities of the initial field and the walls are u / e, the force
increment is g dt / e = g dx / e^2, and the output velocity is e ut.  So for a
loss L on the physical outputs, dL/de follows from the rollout alone; fourth-
order central differences of L in e (with the inputs re-scaled for every e) fix
it independently of the formula.  The sum over the rollout's steps of
nu_term(state_n, lam_(n+1)) -- lam from the oracle's reverse pass -- must equal
e dL/de, with walls (a moving lid), a body force and a loss on rho and u.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs


def _setup(kind):
    g = inputs.rng(81)
    if kind == "channel2d":
        case = inputs.random_case(inputs.D2Q9, (12, 10), 0b01, seed=82, u_amp=0.06, walls="box")
        force_phys = np.array([3e-4, -1e-4])
    elif kind == "cavity2d":
        case = inputs.random_case(inputs.D2Q9, (11, 9), 0b00, seed=83, u_amp=0.06, walls="mixed")
        force_phys = np.array([0.0, 2e-4])
    else:
        case = inputs.random_case(inputs.D3Q19, (6, 5, 7), 0b111, seed=84, u_amp=0.06)
        force_phys = np.array([1e-4, 0.0, -2e-4])
    fluid = ~case.wall_mask if case.node_type is not None else np.ones(case.grid, bool)
    target = 0.05 * g.standard_normal(case.u.shape)
    crho = g.standard_normal(case.grid)
    # physical velocities: the case's lattice velocities at e = 1 (walls included)
    return case, fluid, target, crho, case.u.copy(), force_phys


def _loss(case, fluid, target, crho, u_phys, force_phys, e, steps):
    ut0 = u_phys / e                      # initial and wall velocities u / e
    force = force_phys / (e * e)          # g dt / e with dt = dx / e, dx = 1
    r, ut = orc.step(case.lattice, case.rho, ut0, case.periodic, wall=case.wall_mask, force=force,
                     nsteps=steps)
    uT = e * ut
    return float(np.sum(((uT - target) ** 2)[:, fluid]) + np.sum((crho * r)[fluid])), r, ut


@pytest.mark.parametrize("kind", ["channel2d", "cavity2d", "tgv3d"])
def test_nu_term_sums_to_de_of_loss(kind):
    case, fluid, target, crho, u_phys, force_phys = _setup(kind)
    steps, e = 6, 1.3
    h = 1e-3 * e
    Lf = lambda ee: _loss(case, fluid, target, crho, u_phys, force_phys, ee, steps)[0]
    fd = (8 * (Lf(e + h) - Lf(e - h)) - (Lf(e + 2 * h) - Lf(e - 2 * h))) / (12 * h)
    # states of the rollout at this e, then the reverse pass with the viscosity term
    ut0 = u_phys / e
    force = force_phys / (e * e)
    states = [(case.rho.copy(), ut0.copy())]
    for _ in range(steps):
        states.append(orc.step(case.lattice, *states[-1], case.periodic, wall=case.wall_mask,
                               force=force))
    rT, utT = states[-1]
    lam_r = np.where(fluid, crho, 0.0)
    lam_u = np.where(fluid[None], 2.0 * e * (e * utT - target), 0.0)
    total = 0.0
    for n in range(steps - 1, -1, -1):
        total += orc.nu_term(case.lattice, *states[n], case.periodic, lam_r, lam_u,
                             wall=case.wall_mask, force=force)
        lam_r, lam_u, _ = orc.adjoint_step(case.lattice, *states[n], case.periodic, lam_r, lam_u,
                                           wall=case.wall_mask, force=force)
    assert total == pytest.approx(e * fd, rel=1e-7, abs=1e-12)
