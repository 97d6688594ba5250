"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests runs the CUDA library.  Each one would fail on a plausible
mistake in the oracle (a dropped term, a wrong sign, a wrong weight or index, a
transposed component):

* lattice tables against the lists printed in the paper (tests/golden);
* the moment identities of Eq. (14) and isotropy of the weights;
* exact rational brute force on 4x4 and 4x4x4 grids (walls, wrap, force);
* the tau = 1 reduction of Eq. (1) (Methods): an independent stream-and-collide
  LBM that stores f gives the same (rho, u) on periodic grids; at other tau the
  same comparator (the oracle of the GPU LBM) against an exact rational BGK,
  and its mass and momentum conservation;
* closed forms: Couette Eq. (7) and Couette-Poiseuille Eq. (8) steady states
  (exact at the nodes), the shear-wave and Taylor-Green decay factors, and the
  continuum decay exp(-2 nu k^2 t) of Test 4;
* exact mass and momentum conservation on periodic grids (Eq. (15));
* mirror symmetry of the lid-driven cavities (Tests 3 and 5);
* the adjoint against central finite differences of the forward oracle.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from conftest import read_golden
from oracle import exact_rational, lbm_tau1
from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs

D2, D3 = orc.D2Q9, orc.D3Q19


# ---------------------------------------------------------------- tables, Eq. (14)

def test_lattice_tables_match_paper():
    rows = read_golden("lattices.txt")
    for lat, name in ((D2, "D2Q9"), (D3, "D3Q19")):
        c, w = orc.lattice_table(lat)
        gold = [r for r in rows if r[0] == name]
        assert len(gold) == len(w)
        for r in gold:
            a = int(r[1])
            assert list(c[a]) == [int(r[2]), int(r[3]), int(r[4])]
            assert w[a] == pytest.approx(int(r[5]) / int(r[6]), rel=1e-16)


@pytest.mark.parametrize("lat", [D2, D3])
def test_weight_isotropy(lat):
    c, w = orc.lattice_table(lat)
    d = 2 if lat == D2 else 3
    c = c[:, :d].astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(c.T @ w).max() < 1e-16
    second = np.einsum("a,ai,aj->ij", w, c, c)
    assert np.abs(second - np.eye(d) / 3).max() < 1e-15


@pytest.mark.parametrize("lat", [D2, D3])
def test_equilibrium_moments(lat):
    """Eq. (14): sum_a f^eq = rho and sum_a e_a f^eq = rho u for any (rho, u)."""
    c, _ = orc.lattice_table(lat)
    d = 2 if lat == D2 else 3
    g = inputs.rng(11)
    for _ in range(20):
        rho = 1 + 0.3 * g.uniform(-1, 1)
        ut = 0.4 * g.uniform(-1, 1, size=d)
        f = np.array([orc.feq(lat, a, rho, ut) for a in range(len(c))])
        assert abs(f.sum() - rho) < 1e-15
        assert np.abs(c[:, :d].T @ f - rho * ut).max() < 1e-15


@pytest.mark.parametrize("lat,dims", [(D2, (7, 5)), (D3, (5, 4, 3))])
def test_rest_and_uniform_flow_are_fixed_points(lat, dims):
    d = len(dims)
    grid = tuple(reversed(dims))
    for uval in (0.0, 0.13):
        rho = np.full(grid, 1.07)
        u = np.zeros((d,) + grid)
        u[0] = uval
        u[d - 1] -= 0.5 * uval
        r2, u2 = orc.step(lat, rho, u, (1 << d) - 1, nsteps=3)
        assert np.abs(r2 - rho).max() < 1e-14
        assert np.abs(u2 - u).max() < 1e-15


# ---------------------------------------------------------------- exact rational, 4x4

def _rational_case(d, seed, walls):
    g = inputs.rng(100 + seed)
    dims = (4,) * d
    coords = [tuple(int(v) for v in x) for x in np.ndindex(*dims)]
    rho = {x: Fr(int(g.integers(900, 1100)), 1000) for x in coords}
    u = {x: tuple(Fr(int(g.integers(-60, 61)), 1000) for _ in range(d)) for x in coords}
    wall = set()
    periodic = (1 << d) - 1
    if walls:
        periodic = 0b01 if d == 2 else 0b011            # x (and y) periodic, last axis closed
        wall = {x for x in coords if x[d - 1] in (0, 3)}
        wall |= {coords[int(g.integers(len(coords)))]}  # one interior obstacle
    force = tuple(Fr(int(g.integers(-5, 6)), 10000) for _ in range(d))
    return dims, periodic, rho, u, wall, force


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("walls", [False, True])
def test_exact_rational_bruteforce(d, walls):
    lat = D2 if d == 2 else D3
    dims, periodic, rho, u, wall, force = _rational_case(d, d + 2 * walls, walls)
    grid = tuple(reversed(dims))
    R = np.zeros(grid)
    U = np.zeros((d,) + grid)
    W = np.zeros(grid, dtype=np.uint8)
    for x in rho:
        R[tuple(reversed(x))] = float(rho[x])
        for i in range(d):
            U[(i,) + tuple(reversed(x))] = float(u[x][i])
        W[tuple(reversed(x))] = x in wall
    r_ex, u_ex = rho, u
    r_o, u_o = R, U
    for _ in range(3):
        r_ex, u_ex = exact_rational.step(d, dims, periodic, r_ex, u_ex, wall, force)
        r_o, u_o = orc.step(lat, r_o, u_o, periodic, wall=W if walls else None,
                            force=[float(f) for f in force])
        for x in r_ex:
            ix = tuple(reversed(x))
            assert abs(r_o[ix] - float(r_ex[x])) <= 1e-15 * abs(float(r_ex[x]))
            for i in range(d):
                assert abs(u_o[(i,) + ix] - float(u_ex[x][i])) <= 2e-16 + 1e-14 * abs(float(u_ex[x][i]))


# ---------------------------------------------------------------- tau = 1 reduction

@pytest.mark.parametrize("lat,dims", [(D2, (12, 10)), (D3, (6, 5, 7))])
def test_tau1_stream_collide_equivalence(lat, dims):
    case = inputs.random_case(lat, dims, (1 << len(dims)) - 1, seed=3, u_amp=0.1, rho_amp=0.05)
    _, _, hist = lbm_tau1.run(case.rho, case.u, 6, tau=1.0, record=True)
    r, u = case.rho, case.u
    for n in range(6):
        r, u = orc.step(lat, r, u, case.periodic)
        rh, uh = hist[n]
        assert np.abs(r - rh).max() < 1e-14
        assert np.abs(u - uh).max() < 1e-14


def test_tau1_comparator_differs_at_other_tau():
    """Sanity of the comparator itself: at tau != 1 it is a different scheme."""
    case = inputs.random_case(D2, (8, 8), 0b11, seed=4, u_amp=0.1)
    r1, u1 = lbm_tau1.run(case.rho, case.u, 3, tau=1.0)
    r2, u2 = lbm_tau1.run(case.rho, case.u, 3, tau=0.8)
    assert np.abs(u1 - u2).max() > 1e-4


@pytest.mark.parametrize("tau", [Fr(3, 5), Fr(7, 4)])
def test_bgk_comparator_exact_rational(tau):
    """The general-tau stream-and-collide comparator (the oracle of the GPU
    LBM) against an exact rational BGK on a 4 x 3 periodic grid: a dropped
    term, a wrong sign or a wrong relaxation in the collision would show."""
    rng = np.random.default_rng(7)
    nx, ny = 4, 3
    rho_q = {(x, y): Fr(int(rng.integers(90, 110)), 100) for x in range(nx) for y in range(ny)}
    u_q = {k: (Fr(int(rng.integers(-8, 9)), 100), Fr(int(rng.integers(-8, 9)), 100))
           for k in rho_q}
    rho = np.array([[float(rho_q[(x, y)]) for x in range(nx)] for y in range(ny)])
    u = np.array([[[float(u_q[(x, y)][i]) for x in range(nx)] for y in range(ny)] for i in range(2)])
    r_q, v_q = exact_rational.bgk_run((nx, ny), rho_q, u_q, 3, tau)
    r_f, u_f = lbm_tau1.run(rho, u, 3, tau=float(tau))
    for x in range(nx):
        for y in range(ny):
            assert abs(r_f[y, x] - float(r_q[(x, y)])) < 1e-14
            for i in range(2):
                assert abs(u_f[i, y, x] - float(v_q[(x, y)][i])) < 1e-14


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.6])
def test_bgk_comparator_conserves_mass_and_momentum(tau):
    case = inputs.random_case(D2, (12, 10), 0b11, seed=8, u_amp=0.08, rho_amp=0.03)
    r, u = lbm_tau1.run(case.rho, case.u, 20, tau=tau)
    assert abs(r.sum() - case.rho.sum()) < 1e-11 * case.rho.sum()
    for i in range(2):
        assert abs((r * u[i]).sum() - (case.rho * case.u[i]).sum()) < 1e-12 * case.rho.sum()


# ---------------------------------------------------------------- closed forms

def _channel_steady(u_top_lat, force_x, ny=51, nx=20, nsteps=45000):
    case = inputs.channel2d(nx=nx, ny=ny, u_top=u_top_lat, force_x=force_x)
    r, u = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask,
                    force=case.force, nsteps=nsteps)
    return case, r, u


@pytest.mark.slow
def test_couette_steady_state_is_exact_and_nu_independent():
    """Test 1, Eq. (7): u_x(y) = u0 y / h, whatever nu (three values of the paper)."""
    gold = dict((r[0], r[1:]) for r in read_golden("paper_flows.txt"))
    h, u0, dx = float(gold["test1_h"][0]), float(gold["test1_u0"][0]), float(gold["test1_dx"][0])
    ny = int(gold["test1_ny_spacings"][0]) + 1
    y = np.arange(ny) * dx
    for nu in map(float, gold["test1_nu"]):
        e, _ = orc.params(dx, nu)
        case, r, u = _channel_steady(u0 / e, 0.0, ny=ny)
        ux = u[0] * e                                   # physical
        exact = u0 * y / h
        assert np.abs(ux - exact[:, None]).max() < 1e-12 * u0
        assert np.abs(u[1]).max() < 1e-12 * u0 / e       # rounding only
        assert np.abs(r - 1).max() < 1e-13


@pytest.mark.slow
def test_poiseuille_steady_state_matches_eq8():
    """Test 2, Eq. (8): u(y) = 1/(2 rho nu) dp/dx (y^2 - h y) with both plates fixed."""
    gold = dict((r[0], r[1:]) for r in read_golden("paper_flows.txt"))
    h, dx = float(gold["test1_h"][0]), float(gold["test1_dx"][0])
    dpdx = float(gold["test2_dpdx"][0])
    ny = int(gold["test1_ny_spacings"][0]) + 1
    y = np.arange(ny) * dx
    umax = []
    for nu in map(float, gold["test2_nu"]):
        e, _ = orc.params(dx, nu)
        f_lat = orc.force_lattice([-dpdx, 0.0], dx, nu)
        case, r, u = _channel_steady(0.0, f_lat[0], ny=ny)
        ux = u[0] * e
        exact = dpdx / (2 * 1.0 * nu) * (y ** 2 - h * y)
        # FP64 floor: the x-momentum sum cancels O(0.1) terms (rounding ~1e-17 per
        # step), which the steady balance amplifies by ~6 H^2 / 8: ~3e-14 lattice
        assert np.abs(ux - exact[:, None]).max() < 1e-13 * e
        umax.append(ux.max())
    # centre-line speeds implied by Eq. (8) for the paper's three viscosities
    assert umax == pytest.approx([1e-4 / (8 * nu) for nu in (0.003, 0.001, 0.0006)], rel=1e-10)


@pytest.mark.parametrize("lat", [D2, D3])
def test_shear_wave_decays_exactly(lat):
    """A shear wave u_x = A sin(k y) keeps its shape and decays by (2 + cos k)/3 per
    step at any amplitude: the equilibrium's quadratic terms cancel in Eqs. (4)-(5)
    for a unidirectional flow, and what remains is a 3-point average."""
    d = 2 if lat == D2 else 3
    n = 16
    dims = (4, n) if d == 2 else (4, n, 3)
    grid = tuple(reversed(dims))
    k = 2 * math.pi / n
    yy = np.arange(n) * k
    A = 0.3
    u = np.zeros((d,) + grid)
    shape = [1] * d
    shape[d - 2] = n
    u[0] = A * np.sin(yy).reshape(shape)
    rho = np.ones(grid)
    steps = 100
    r, u2 = orc.step(lat, rho, u, (1 << d) - 1, nsteps=steps)
    G = (2 + math.cos(k)) / 3
    assert np.abs(u2[0] - G ** steps * u[0]).max() < 1e-13 * A
    assert np.abs(u2[1:]).max() < 1e-15
    assert np.abs(r - 1).max() < 1e-14


def test_tgv2d_discrete_and_continuum_decay():
    """Test 4 mode on 64^2: per-step factor (1 + 2 cos k)/3 from linearising
    Eqs. (4)-(5); its continuum limit is exp(-2 nu k^2 dt) with nu dt / dx^2 = 1/6."""
    n, steps = 64, 1000
    k = 2 * math.pi / n
    G = (1 + 2 * math.cos(k)) / 3
    for u0, tol in ((1e-4, 1e-9), (0.02, 1e-5)):
        case = inputs.tgv2d(n, u0)
        r, u = orc.step(D2, case.rho, case.u, case.periodic, nsteps=steps)
        amp = np.sum(u * case.u) / np.sum(case.u * case.u)
        assert amp == pytest.approx(G ** steps, rel=tol)
    # continuum: e = 1, dx = 1, nu = 1/6, dt = 1
    assert amp == pytest.approx(math.exp(-2 * (1 / 6) * k * k * steps), rel=5e-3)


def test_tgv3d_discrete_decay():
    """Standard 3D TGV mode on D3Q19: per-step factor (1 + cos k + cos^2 k)/3."""
    n, steps = 16, 40
    k = 2 * math.pi / n
    G = (1 + math.cos(k) + math.cos(k) ** 2) / 3
    case = inputs.tgv3d(n, 1e-5)
    r, u = orc.step(D3, case.rho, case.u, case.periodic, nsteps=steps)
    amp = np.sum(u * case.u) / np.sum(case.u * case.u)
    assert amp == pytest.approx(G ** steps, rel=1e-8)


def test_paper_tgv_setup_decay():
    """Test 4 as printed: 40 x 40 over 2 pi, nu = 0.0314, u0 = 0.05, t = 30 s;
    the amplitude must follow exp(-2 nu t) (k = 1) within the O(dx^2) error."""
    gold = dict((r[0], r[1:]) for r in read_golden("paper_flows.txt"))
    n = int(gold["test4_n"][0])
    nu, u0, t_end = float(gold["test4_nu"][0]), float(gold["test4_u0"][0]), float(gold["test4_t"][0])
    dx = 2 * math.pi / n                   # 0.157 is this value rounded
    e, dt = orc.params(dx, nu)
    steps = round(t_end / dt)
    case = inputs.tgv2d(n, u0 / e)
    r, u = orc.step(D2, case.rho, case.u, case.periodic, nsteps=steps)
    amp = np.sum(u * case.u) / np.sum(case.u * case.u)
    assert amp == pytest.approx(math.exp(-2 * nu * steps * dt), rel=2e-2)


# ---------------------------------------------------------------- conservation, symmetry

@pytest.mark.parametrize("lat,dims", [(D2, (24, 17)), (D3, (9, 8, 7))])
def test_periodic_conservation(lat, dims):
    """Eq. (15): total mass and momentum are invariants of the periodic update."""
    case = inputs.random_case(lat, dims, (1 << len(dims)) - 1, seed=7, u_amp=0.1, rho_amp=0.05)
    d0 = orc.diagnostics(case.rho, case.u)
    r, u = orc.step(lat, case.rho, case.u, case.periodic, nsteps=200)
    d1 = orc.diagnostics(r, u)
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-13)
    for i in range(len(dims)):
        assert abs(d1["momentum"][i] - d0["momentum"][i]) < 1e-13 * d0["mass"]


def test_cavity2d_mirror_symmetry():
    """Reflecting x and reversing the lid maps the 2D cavity solution to itself."""
    n = 24
    a = inputs.cavity2d(n, lid=0.1)
    b = inputs.cavity2d(n, lid=-0.1)
    ra, ua = orc.step(D2, a.rho, a.u, 0, wall=a.wall_mask, nsteps=150)
    rb, ub = orc.step(D2, b.rho, b.u, 0, wall=b.wall_mask, nsteps=150)
    assert np.abs(rb - ra[:, ::-1]).max() < 1e-13
    assert np.abs(ub[0] + ua[0][:, ::-1]).max() < 1e-13
    assert np.abs(ub[1] - ua[1][:, ::-1]).max() < 1e-13
    assert np.abs(ua[1]).max() > 1e-3      # the flow is genuinely 2D


def test_cavity3d_spanwise_symmetry():
    """3D cavity, lid along +x: reflecting y leaves u_x, u_z even and u_y odd."""
    n = 12
    c = inputs.cavity3d(n, lid=0.1)
    r, u = orc.step(D3, c.rho, c.u, 0, wall=c.wall_mask, nsteps=60)
    assert np.abs(r - r[:, ::-1, :]).max() < 1e-13
    assert np.abs(u[0] - u[0][:, ::-1, :]).max() < 1e-13
    assert np.abs(u[2] - u[2][:, ::-1, :]).max() < 1e-13
    assert np.abs(u[1] + u[1][:, ::-1, :]).max() < 1e-13
    assert np.abs(u[2]).max() > 1e-3


def test_open_boundary_is_rejected():
    case = inputs.random_case(D2, (6, 6), 0b01, seed=1)   # y closed but no walls
    with pytest.raises(ValueError):
        orc.step(D2, case.rho, case.u, case.periodic)


# ---------------------------------------------------------------- adjoint

def _loss_grad_fd(lat, case, steps, v_r, v_u, w_r, w_u, eps=1e-6):
    """<J v, w> by central differences of the forward oracle."""
    def fwd(s):
        return orc.step(lat, case.rho + s * v_r, case.u + s * v_u, case.periodic,
                        wall=case.wall_mask, force=case.force, nsteps=steps)
    rp, up = fwd(eps)
    rm, um = fwd(-eps)
    return (np.sum((rp - rm) * w_r) + np.sum((up - um) * w_u)) / (2 * eps)


@pytest.mark.parametrize("lat,dims,walls,periodic", [
    (D2, (9, 8), "none", 0b11), (D2, (10, 9), "mixed", 0b01),
    (D3, (6, 5, 6), "none", 0b111), (D3, (6, 6, 5), "box", 0b011)])
def test_adjoint_dot_product(lat, dims, walls, periodic):
    d = len(dims)
    case = inputs.random_case(lat, dims, periodic, seed=21, u_amp=0.08, walls=walls,
                              force=tuple([2e-4] * d))
    g = inputs.rng(22)
    v_r = g.standard_normal(case.rho.shape)
    v_u = g.standard_normal(case.u.shape)
    if case.wall_mask is not None:        # wall values are parameters, not state
        v_r[case.wall_mask] = 0
        v_u[:, case.wall_mask] = 0
    w_r = g.standard_normal(case.rho.shape)
    w_u = g.standard_normal(case.u.shape)
    steps = 10
    jvp = _loss_grad_fd(lat, case, steps, v_r, v_u, w_r, w_u)
    lr, lu, gf = orc.rollout_adjoint(lat, case.rho, case.u, periodic, steps, w_r, w_u,
                                     wall=case.wall_mask, force=case.force)
    vjp = np.sum(lr * v_r) + np.sum(lu * v_u)
    assert vjp == pytest.approx(jvp, rel=1e-7)
    # force gradient by central differences
    eps = 1e-7
    for i in range(d):
        fp = list(case.force); fp[i] += eps
        fm = list(case.force); fm[i] -= eps
        rp, up = orc.step(lat, case.rho, case.u, periodic, wall=case.wall_mask, force=fp,
                          nsteps=steps)
        rm, um = orc.step(lat, case.rho, case.u, periodic, wall=case.wall_mask, force=fm,
                          nsteps=steps)
        fd = (np.sum((rp - rm) * w_r) + np.sum((up - um) * w_u)) / (2 * eps)
        assert gf[i] == pytest.approx(fd, rel=1e-6)


def test_adjoint_wall_value_gradient():
    """Gradient w.r.t. a wall id's velocity = sum of the initial-state adjoint over
    its nodes (the wall value is copied into every step), checked by differences."""
    case = inputs.random_case(D2, (10, 9), 0b01, seed=23, u_amp=0.08, walls="box")
    g = inputs.rng(24)
    w_r = g.standard_normal(case.rho.shape)
    w_u = g.standard_normal(case.u.shape)
    steps = 8
    lr, lu, _ = orc.rollout_adjoint(D2, case.rho, case.u, case.periodic, steps, w_r, w_u,
                                    wall=case.wall_mask)
    for k in (1, 2):
        sel = case.node_type == k
        eps = 1e-6
        vals = []
        for s in (eps, -eps):
            wu = case.wall_u.copy()
            wu[k - 1, 0] += s
            r0, u0 = inputs.place_walls(case.rho, case.u, case.node_type, case.wall_rho, wu)
            r1, u1 = orc.step(D2, r0, u0, case.periodic, wall=case.wall_mask, nsteps=steps)
            vals.append(np.sum(r1 * w_r) + np.sum(u1 * w_u))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert np.sum(lu[0][sel]) == pytest.approx(fd, rel=1e-7)


def test_params_eq6():
    e, dt = orc.params(0.02, 0.001)
    assert e == pytest.approx(0.3, rel=1e-15)
    assert dt == pytest.approx(0.02 / 0.3, rel=1e-15)
    assert dt == pytest.approx(0.02 ** 2 / (6 * 0.001), rel=1e-14)
    # R_le = U dx / nu = 6 U / e: the lattice Mach number times six
    assert orc.lattice_reynolds(0.1, 0.02, 0.001) == pytest.approx(6 * 0.1 / e, rel=1e-14)


def test_diagnostics_hand_computed():
    """The FP64 diagnostics on a 2 x 2 field worked out by hand (values chosen
    so every sum is exact in binary); the wall node, with large values, must
    not count."""
    rho = np.array([[1.0, 2.0], [0.5, 4.0]])                    # [y, x]
    u = np.array([[[0.5, -0.25], [1.0, 3.0]],                   # u_x
                  [[0.0, 0.5], [-0.5, 7.0]]])                   # u_y
    fluid = np.array([[True, True], [True, False]])             # node (y=1, x=1) is a wall
    d = orc.diagnostics(rho, u, u_prev=0.5 * u, fluid=fluid)
    # mass 1 + 2 + 0.5; kinetic 1/2 (1*0.25 + 2*(0.0625 + 0.25) + 0.5*(1 + 0.25))
    assert d["mass"] == 3.5
    assert d["kinetic"] == 0.75
    # momentum: x 0.5 - 0.5 + 0.5, y 0 + 1 - 0.25
    assert d["momentum"] == [0.5, 0.75]
    # u - u_prev = u / 2 on the fluid nodes
    assert d["residual"] == pytest.approx(0.5, rel=1e-15)
    assert orc.diagnostics(rho, u, u_prev=u, fluid=fluid)["residual"] == 0.0
