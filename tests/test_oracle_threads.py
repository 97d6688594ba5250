"""The oracle's host threads change no result.

The FP64 oracle runs its node loops on several host threads (OpenMP) so that
long runs of the paper's workloads can be checked against it at full size.
Each value is still formed by one thread with the single-thread operations in
the single-thread order, so the results must be bitwise equal to one thread's:

* the forward step (Eqs. (4)-(5)) at 1 thread and at all cores;
* the adjoint written as a gather over sources against the plain scatter of
  the chain rule (one thread), including grids of one and two nodes along a
  periodic axis, where several directions of one source reach the same node;
* a checkpointed reverse pass (states recomputed from every K-th state)
  against the one that stores every state.

These run on the CPU only.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs

D2, D3 = orc.D2Q9, orc.D3Q19

CASES = [
    (D2, (13, 11), 0b01, "box"),
    (D2, (9, 7), 0b11, "none"),
    (D2, (2, 5), 0b11, "none"),      # two nodes along x: +x and -x reach the same node
    (D2, (1, 6), 0b11, "none"),      # one node along x
    (D2, (12, 10), 0b00, "mixed"),
    (D3, (10, 9, 8), 0b101, "box"),
    (D3, (7, 6, 5), 0b111, "none"),
    (D3, (2, 3, 2), 0b111, "none"),
    (D3, (9, 8, 7), 0b000, "mixed"),
]


@pytest.fixture(autouse=True)
def _restore_threads():
    n = orc.set_threads(0)
    yield
    orc.set_threads(n)


@pytest.mark.parametrize("lat,dims,periodic,walls", CASES)
def test_forward_threads_bitwise(lat, dims, periodic, walls):
    case = inputs.random_case(lat, dims, periodic, seed=11, u_amp=0.08, walls=walls)
    force = [1e-4, -2e-5, 3e-5][: case.d]
    orc.set_threads(1)
    r1, u1 = orc.step(lat, case.rho, case.u, periodic, wall=case.wall_mask, force=force, nsteps=4)
    orc.set_threads(max(2, orc.host_cores()))
    rn, un = orc.step(lat, case.rho, case.u, periodic, wall=case.wall_mask, force=force, nsteps=4)
    assert np.array_equal(r1, rn) and np.array_equal(u1, un)


@pytest.mark.parametrize("lat,dims,periodic,walls", CASES)
def test_adjoint_gather_equals_scatter_bitwise(lat, dims, periodic, walls):
    case = inputs.random_case(lat, dims, periodic, seed=12, u_amp=0.08, walls=walls)
    g = np.random.default_rng(5)
    lr = g.standard_normal(case.rho.shape)
    lu = g.standard_normal(case.u.shape)
    force = [1e-4, -2e-5, 3e-5][: case.d]
    orc.set_threads(1)
    a = orc.adjoint_step(lat, case.rho, case.u, periodic, lr, lu, wall=case.wall_mask, force=force)
    orc.set_threads(max(2, orc.host_cores()))
    b = orc.adjoint_step(lat, case.rho, case.u, periodic, lr, lu, wall=case.wall_mask, force=force,
                         gather=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # the plain scatter itself does not depend on the thread count either
    c = orc.adjoint_step(lat, case.rho, case.u, periodic, lr, lu, wall=case.wall_mask, force=force)
    for x, y in zip(a, c):
        assert np.array_equal(x, y)


def test_adjoint_gather_reports_open_boundary():
    case = inputs.random_case(D2, (6, 5), 0b00, seed=1, walls="none")
    lr = np.ones(case.rho.shape)
    lu = np.ones(case.u.shape)
    with pytest.raises(ValueError):
        orc.adjoint_step(D2, case.rho, case.u, 0b00, lr, lu, gather=True)
    with pytest.raises(ValueError):
        orc.adjoint_step(D2, case.rho, case.u, 0b00, lr, lu)


@pytest.mark.parametrize("lat,dims,periodic,walls", [CASES[0], CASES[5]])
@pytest.mark.parametrize("every", [1, 3, 4, 7])
def test_checkpointed_rollout_bitwise(lat, dims, periodic, walls, every):
    case = inputs.random_case(lat, dims, periodic, seed=13, u_amp=0.06, walls=walls)
    g = np.random.default_rng(6)
    lr = g.standard_normal(case.rho.shape)
    lu = g.standard_normal(case.u.shape)
    force = [2e-5, 1e-5, -1e-5][: case.d]
    ref = orc.rollout_adjoint(lat, case.rho, case.u, periodic, 10, lr, lu, wall=case.wall_mask,
                              force=force)
    got = orc.rollout_adjoint(lat, case.rho, case.u, periodic, 10, lr, lu, wall=case.wall_mask,
                              force=force, checkpoint_every=every, gather=True)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
