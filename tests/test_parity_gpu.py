"""GPU parity: the CUDA step (through the C ABI) against the FP64 CPU oracle.

Same seeded inputs on both sides; element-wise comparison.  Bars:
  * FP64 storage: <= 1e-12 relative (max norm) on rho and u;
  * FP32 storage: <= 1e-5 relative L2 on u, <= 1e-6 absolute on rho;
  * BF16 / FP16 storage (FP32 arithmetic): the error is stated, not held to
    1e-5: <= 2e-2 (bf16) and <= 3e-3 (f16) relative L2 on u after 7 steps.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu

D2, D3 = inputs.D2Q9, inputs.D3Q19
TOL_U = {M.F64: 1e-12, M.F32: 1e-5, M.BF16_STORE: 2e-2, M.F16_STORE: 3e-3}
TOL_R = {M.F64: 1e-12, M.F32: 1e-6, M.BF16_STORE: 1e-3, M.F16_STORE: 2e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


def rel_l2(a, b):
    nb = np.sqrt(np.sum(b * b))
    return np.sqrt(np.sum((a - b) ** 2)) / (nb if nb > 0 else 1.0)


def run_both(case, precision, steps, kernel=None):
    s = M.Solver.from_case(case, precision)
    if kernel is not None:
        s.set_kernel(kernel)
    s.step(steps)
    r_g, u_g = s.get_state()
    s.close()
    r_o, u_o = orc.step(case.lattice, case.rho, case.u, case.periodic, wall=case.wall_mask,
                        force=case.force, nsteps=steps)
    return r_g, u_g, r_o, u_o


def assert_parity(r_g, u_g, r_o, u_o, precision):
    if precision == M.F64:
        assert np.abs(r_g - r_o).max() <= TOL_R[precision] * np.abs(r_o).max()
        assert np.abs(u_g - u_o).max() <= TOL_U[precision] * max(np.abs(u_o).max(), 1e-300)
    else:
        assert np.abs(r_g - r_o).max() <= TOL_R[precision]
        assert rel_l2(u_g, u_o) <= TOL_U[precision]


CASES = [
    # lattice, dims, periodic, walls
    (D2, (17, 13), 0b11, "none"),
    (D2, (33, 20), 0b00, "box"),
    (D2, (40, 23), 0b01, "mixed"),
    (D3, (9, 7, 5), 0b111, "none"),
    (D3, (12, 10, 9), 0b000, "box"),
    (D3, (16, 9, 11), 0b101, "mixed"),
]


@pytest.mark.parametrize("lat,dims,periodic,walls", CASES)
@pytest.mark.parametrize("precision", [M.F64, M.F32])
@pytest.mark.parametrize("steps", [1, 7])
def test_random_fields(lat, dims, periodic, walls, precision, steps):
    case = inputs.random_case(lat, dims, periodic, seed=31, u_amp=0.08, rho_amp=0.02,
                              walls=walls, force=tuple([1e-4] * len(dims)))
    assert_parity(*run_both(case, precision, steps), precision)


# Sizes the tiled kernel serves (x a multiple of 4), with ragged tiles in y and
# the march axis, every wall mode and several periodicities.
TILED_CASES = [
    (D2, (16, 13), 0b11, "none"),
    (D2, (64, 37), 0b00, "box"),
    (D2, (96, 41), 0b01, "mixed"),
    (D2, (4, 9), 0b11, "none"),
    (D2, (256, 70), 0b10, "box"),
    (D3, (8, 8, 5), 0b111, "none"),
    (D3, (12, 10, 9), 0b000, "box"),
    (D3, (16, 9, 19), 0b101, "mixed"),
    (D3, (32, 16, 7), 0b011, "box"),
    (D3, (4, 8, 3), 0b111, "none"),
    (D3, (20, 13, 17), 0b100, "mixed"),
]


@pytest.mark.parametrize("lat,dims,periodic,walls", TILED_CASES)
@pytest.mark.parametrize("precision", [M.F64, M.F32, M.BF16_STORE])
@pytest.mark.parametrize("steps", [1, 5])
def test_tiled_kernel(lat, dims, periodic, walls, precision, steps):
    case = inputs.random_case(lat, dims, periodic, seed=37, u_amp=0.08, rho_amp=0.02,
                              walls=walls, force=tuple([-2e-4] * len(dims)))
    s = M.Solver.from_case(case, precision)
    try:
        s.set_kernel(M.KERNEL_TILED)
    except M.MacLABError as e:
        s.close()
        # FP32 is built for every width; FP64 / 16-bit storage only for some
        assert precision != M.F32 and e.status == M.ERR_UNSUPPORTED
        pytest.skip("no tiled instance of this width for this storage type")
    assert s.kernel_info()["kernel"] == M.KERNEL_TILED
    s.close()
    assert_parity(*run_both(case, precision, steps, kernel=M.KERNEL_TILED), precision)


@pytest.mark.parametrize("lat,dims,periodic,walls", TILED_CASES)
def test_tiled_matches_reference_kernel(lat, dims, periodic, walls):
    """The two kernels compute the same sums in a different order: FP32 results
    agree to rounding (a few ulp of |u| per step)."""
    case = inputs.random_case(lat, dims, periodic, seed=38, u_amp=0.08, rho_amp=0.02, walls=walls)
    out = []
    for kern in (M.KERNEL_REFERENCE, M.KERNEL_TILED):
        s = M.Solver.from_case(case, M.F32)
        s.set_kernel(kern)
        s.step(10)
        out.append(s.get_state())
        s.close()
    (r1, u1), (r2, u2) = out
    assert np.abs(r1 - r2).max() < 1e-6
    assert np.abs(u1 - u2).max() < 2e-6 * np.abs(u1).max()


# The folded D3Q19 kernel (no halo-row threads): FP32, x a multiple of 4 up to
# 512, ny a multiple of the tile's rows; one-tile y extents wrap onto themselves.
FOLD_CASES = [
    ((8, 8, 5), 0b111, "none", 0),
    ((12, 8, 9), 0b000, "box", 0),
    ((16, 16, 19), 0b101, "mixed", 0),
    ((32, 16, 7), 0b011, "box", 0),
    ((128, 8, 6), 0b000, "box", 0),
    ((96, 12, 10), 0b010, "mixed", 0),
    ((256, 8, 5), 0b111, "none", 0),
    ((4, 8, 3), 0b111, "none", 0),
    ((20, 16, 17), 0b100, "mixed", 0),
    ((128, 4, 9), 0b111, "none", 0),
    ((128, 16, 11), 0b000, "box", 8),
    ((64, 24, 13), 0b110, "mixed", 8),
    ((512, 8, 4), 0b000, "box", 0),
    ((256, 16, 5), 0b101, "mixed", 8),
    ((4, 8, 6), 0b000, "box", 0),       # one quad per row: both x-walls in one lane
    ((8, 16, 7), 0b010, "box", 0),      # two lanes, one x-wall each
]


@pytest.mark.parametrize("dims,periodic,walls,ty", FOLD_CASES)
@pytest.mark.parametrize("steps", [1, 5])
def test_folded_kernel(dims, periodic, walls, ty, steps):
    case = inputs.random_case(D3, dims, periodic, seed=41, u_amp=0.08, rho_amp=0.02,
                              walls=walls, force=(1e-4, -2e-4, 3e-4))
    s = M.Solver.from_case(case, M.F32)
    s.set_kernel(M.KERNEL_FOLDED)
    if ty:
        s.set_tile(ty, 0)
    assert s.kernel_info()["kernel"] == M.KERNEL_FOLDED
    s.step(steps)
    r_g, u_g = s.get_state()
    s.close()
    r_o, u_o = orc.step(D3, case.rho, case.u, case.periodic, wall=case.wall_mask,
                        force=case.force, nsteps=steps)
    assert_parity(r_g, u_g, r_o, u_o, M.F32)


@pytest.mark.parametrize("dims,periodic,walls,ty", FOLD_CASES)
def test_folded_matches_tiled_kernel(dims, periodic, walls, ty):
    """Same terms, summed in another order: FP32 results agree to rounding."""
    case = inputs.random_case(D3, dims, periodic, seed=42, u_amp=0.08, rho_amp=0.02, walls=walls)
    out = []
    for kern in (M.KERNEL_TILED, M.KERNEL_FOLDED):
        s = M.Solver.from_case(case, M.F32)
        s.set_kernel(kern)
        s.step(10)
        out.append(s.get_state())
        s.close()
    (r1, u1), (r2, u2) = out
    assert np.abs(r1 - r2).max() < 1e-6
    assert np.abs(u1 - u2).max() < 2e-6 * np.abs(u1).max()


@pytest.mark.parametrize("precision", [M.BF16_STORE, M.F16_STORE])
@pytest.mark.parametrize("dims,periodic,walls,ty", [((128, 8, 6), 0b000, "box", 0),
                                                    ((96, 12, 10), 0b010, "mixed", 0),
                                                    ((128, 16, 11), 0b000, "box", 8),
                                                    ((256, 8, 5), 0b111, "none", 0)])
def test_folded_kernel_16bit_storage(precision, dims, periodic, walls, ty):
    """16-bit storage, FP32 arithmetic: the oracle within the stated storage
    error, and the tiled kernel within one rounding of the stored value."""
    case = inputs.random_case(D3, dims, periodic, seed=49, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=(1e-4, -2e-4, 3e-4))
    out = []
    for kern in (M.KERNEL_FOLDED, M.KERNEL_TILED):
        s = M.Solver.from_case(case, precision)
        s.set_kernel(kern)
        if ty and kern == M.KERNEL_FOLDED:
            s.set_tile(ty, 0)
        assert s.kernel_info()["kernel"] == kern
        s.step(7)
        out.append(s.get_state())
        s.close()
    (r_f, u_f), (r_t, u_t) = out
    r_o, u_o = orc.step(D3, case.rho, case.u, case.periodic, wall=case.wall_mask, force=case.force,
                        nsteps=7)
    assert_parity(r_f, u_f, r_o, u_o, precision)
    ulp = 2.0 ** -8 if precision == M.BF16_STORE else 2.0 ** -11
    assert np.abs(u_f - u_t).max() <= 4 * ulp * np.abs(u_t).max()
    assert np.abs(r_f - r_t).max() <= 4 * ulp * 0.05


@pytest.mark.parametrize("precision", [M.BF16_STORE, M.F16_STORE])
@pytest.mark.parametrize("dims,periodic,walls", [((400, 8, 6), 0b000, "box"), ((512, 4, 5), 0b111, "none"),
                                                 ((272, 12, 5), 0b010, "mixed")])
def test_folded_kernel_16bit_wide_rows(precision, dims, periodic, walls):
    """Rows of 65 to 128 quads (up to 512 nodes) in 16-bit storage run the
    folded kernel by default (no tiled instance serves them), within the
    stated storage error against the oracle."""
    case = inputs.random_case(D3, dims, periodic, seed=56, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=(1e-4, 0.0, -1e-4))
    s = M.Solver.from_case(case, precision)
    assert s.kernel_info()["kernel"] == M.KERNEL_FOLDED
    s.step(7)
    r_g, u_g = s.get_state()
    s.close()
    r_o, u_o = orc.step(D3, case.rho, case.u, case.periodic, wall=case.wall_mask, force=case.force,
                        nsteps=7)
    assert_parity(r_g, u_g, r_o, u_o, precision)


@pytest.mark.parametrize("precision,dims", [(M.F64, (32, 8, 5)), (M.F32, (32, 6, 5)),
                                            (M.F32, (16, 12, 5)), (M.BF16_STORE, (16, 8, 5))])
def test_folded_rejects_unsupported(precision, dims):
    case = inputs.random_case(D3, dims, 0b111, seed=43)
    s = M.Solver.from_case(case, precision)
    before = s.kernel_info()["kernel"]
    with pytest.raises(M.MacLABError) as ei:
        s.set_kernel(M.KERNEL_FOLDED)
    assert ei.value.status == M.ERR_UNSUPPORTED
    assert s.kernel_info()["kernel"] == before
    s.close()


# The segment kernel (the batched D2Q9 kernel on one domain) for every width it
# serves, tz = rows per work item.
SEG_CASES = [
    ((16, 13), 0b11, "none", 0),
    ((64, 37), 0b00, "box", 2),
    ((96, 41), 0b01, "mixed", 4),
    ((4, 9), 0b11, "none", 16),
    ((256, 70), 0b10, "box", 3),
    ((248, 33), 0b11, "mixed", 0),
    ((4, 9), 0b00, "box", 2),           # one quad per row: both x-walls in one lane
    ((8, 12), 0b10, "box", 3),          # two lanes, one x-wall each
]


@pytest.mark.parametrize("dims,periodic,walls,rows", SEG_CASES)
@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_segment_kernel(dims, periodic, walls, rows, precision):
    case = inputs.random_case(D2, dims, periodic, seed=44, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=(1e-4, -2e-4))
    s = M.Solver.from_case(case, precision)
    s.set_kernel(M.KERNEL_SEGMENT)
    s.set_tile(0, rows)
    assert s.kernel_info()["kernel"] == M.KERNEL_SEGMENT
    s.step(7)
    r_g, u_g = s.get_state()
    x = s.get_lattice_state().copy()
    s.close()
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask, force=case.force,
                        nsteps=7)
    assert_parity(r_g, u_g, r_o, u_o, precision)
    # the same bits as the tiled kernel
    t = M.Solver.from_case(case, precision)
    t.set_kernel(M.KERNEL_TILED)
    t.step(7)
    assert np.array_equal(t.get_lattice_state(), x)
    t.close()


@pytest.mark.parametrize("precision", [M.F64, M.F32])
@pytest.mark.parametrize("steps", [1, 2, 9, 40, 67])
@pytest.mark.parametrize("dims,periodic,walls", [((136, 45), 0b01, "mixed"), ((136, 45), 0b00, "box"),
                                                 ((8, 12), 0b10, "box")])
def test_segment_two_steps_per_launch(precision, steps, dims, periodic, walls):
    """ty = 2: two updates per launch on one domain, runs of n steps ending in a
    one-step launch; the same bits and the same residual as the tiled kernel."""
    case = inputs.random_case(D2, dims, periodic, seed=48, u_amp=0.05, walls=walls,
                              force=(1e-4, 0.0))
    s = M.Solver.from_case(case, precision)
    s.set_kernel(M.KERNEL_SEGMENT)
    s.set_tile(2, 4)
    assert s.kernel_info()["steps_per_launch"] == 2
    s.step(steps)
    t = M.Solver.from_case(case, precision)
    t.set_kernel(M.KERNEL_TILED)
    t.step(steps)
    assert np.array_equal(s.get_lattice_state(), t.get_lattice_state())
    assert s.diagnostics()["residual"] == t.diagnostics()["residual"]
    assert s.params["steps"] == steps
    s.close()
    t.close()


@pytest.mark.parametrize("precision", [M.F64, M.F32])
@pytest.mark.parametrize("steps", [1, 2, 9, 131])
@pytest.mark.parametrize("dims,periodic,walls,rows", [((136, 45), 0b01, "mixed", 2), ((256, 256), 0b00, "box", 2),
                                                      ((8, 12), 0b10, "box", 4), ((64, 64), 0b11, "none", 8)])
def test_segment_persistent(precision, steps, dims, periodic, walls, rows):
    """ty = 3: the step pairs of a run in one persistent cooperative launch,
    each block waiting between sweeps for the blocks that own rows within two
    of its own instead of a kernel boundary; runs end in a one-step launch.
    The same bits as the tiled kernel, across calls, and no wait ran out
    (maclab_sync)."""
    case = inputs.random_case(D2, dims, periodic, seed=49, u_amp=0.05, walls=walls,
                              force=(1e-4, -1e-4))
    s = M.Solver.from_case(case, precision)
    s.set_kernel(M.KERNEL_SEGMENT)
    s.set_tile(3, rows)
    assert s.kernel_info()["steps_per_launch"] == 2
    s.step(steps)
    s.step(steps + 3)
    s.sync()
    t = M.Solver.from_case(case, precision)
    t.set_kernel(M.KERNEL_TILED)
    t.step(2 * steps + 3)
    assert np.array_equal(s.get_lattice_state(), t.get_lattice_state())
    assert s.diagnostics()["residual"] == t.diagnostics()["residual"]
    s.close()
    t.close()


def test_segment_persistent_wait_runs_out():
    """A zero wait budget makes the persistent launch's first wait between
    blocks give up at once: the blocks end their sweeps, the next sync reports
    MACLAB_ERR_TIMEOUT (and only that one), and the context stays usable -- a
    fresh set_state with the default budget gives the tiled kernel's bits."""
    case = inputs.random_case(D2, (256, 256), 0b00, seed=50, u_amp=0.05, walls="box")
    s = M.Solver.from_case(case, M.F32)
    s.set_kernel(M.KERNEL_SEGMENT)
    s.set_tile(3, 2)
    s.set_wait_limit(0)
    s.step(10)
    with pytest.raises(M.MacLABError) as e:
        s.sync()
    assert e.value.status == M.ERR_TIMEOUT
    s.sync()  # the status word was cleared
    s.set_wait_limit(-1)
    s.set_state(np.asarray(case.rho, np.float64), np.asarray(case.u, np.float64))  # e = 1
    s.step(10)
    s.sync()
    t = M.Solver.from_case(case, M.F32)
    t.set_kernel(M.KERNEL_TILED)
    t.step(10)
    assert np.array_equal(s.get_lattice_state(), t.get_lattice_state())
    s.close()
    t.close()


def test_segment_default_for_large_2d_and_graphs():
    """1024^2 picks the segment kernel; 40 steps (a 32-step graph and 8
    launches) equal the tiled kernel's bits; a change of rows per item
    rebuilds the work list and keeps the result."""
    case = inputs.random_case(D2, (1024, 1024), 0b00, seed=45, u_amp=0.05, walls="box")
    s = M.Solver.from_case(case, M.F32)
    assert s.kernel_info()["kernel"] == M.KERNEL_SEGMENT
    s.step(20)
    s.set_tile(0, 8)
    s.step(20)
    t = M.Solver.from_case(case, M.F32)
    t.set_kernel(M.KERNEL_TILED)
    t.step(40)
    assert np.array_equal(s.get_lattice_state(), t.get_lattice_state())
    s.close()
    t.close()


def test_segment_large_2d_two_steps_per_launch():
    """Above 524,288 quads (here 2048^2) the default is two steps per launch
    with 32 rows per work item: 5 steps against the oracle over the whole
    field, and 9 steps bit for bit against one step per launch."""
    case = inputs.random_case(D2, (2048, 2048), 0b00, seed=57, u_amp=0.08, rho_amp=0.02, walls="box")
    s = M.Solver.from_case(case, M.F32)
    info = s.kernel_info()
    assert info["kernel"] == M.KERNEL_SEGMENT and info["steps_per_launch"] == 2
    s.step(5)
    r_g, u_g = s.get_state()
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask, nsteps=5)
    assert_parity(r_g, u_g, r_o, u_o, M.F32)
    s.step(4)
    x = s.get_lattice_state().copy()
    s.close()
    t = M.Solver.from_case(case, M.F32)
    t.set_tile(1, 4)
    assert t.kernel_info()["steps_per_launch"] == 1
    t.step(9)
    assert np.array_equal(t.get_lattice_state(), x)
    t.close()


def test_segment_rejects_3d_and_odd_widths():
    for case in (inputs.random_case(D3, (8, 8, 8), 0b111, seed=46),
                 inputs.random_case(D2, (17, 13), 0b11, seed=47)):
        s = M.Solver.from_case(case, M.F32)
        before = s.kernel_info()["kernel"]
        with pytest.raises(M.MacLABError) as ei:
            s.set_kernel(M.KERNEL_SEGMENT)
        assert ei.value.status == M.ERR_UNSUPPORTED
        assert s.kernel_info()["kernel"] == before
        s.close()


def test_tiled_rejects_unsupported_shape():
    case = inputs.random_case(D2, (17, 13), 0b11, seed=39)
    s = M.Solver.from_case(case, M.F32)
    with pytest.raises(M.MacLABError) as ei:
        s.set_kernel(M.KERNEL_TILED)
    assert ei.value.status == M.ERR_UNSUPPORTED
    assert s.kernel_info()["kernel"] == M.KERNEL_REFERENCE
    s.close()


@pytest.mark.parametrize("lat,dims,periodic,walls", [CASES[1], CASES[4]])
@pytest.mark.parametrize("precision", [M.BF16_STORE, M.F16_STORE])
def test_16bit_storage(lat, dims, periodic, walls, precision):
    case = inputs.random_case(lat, dims, periodic, seed=32, u_amp=0.08, rho_amp=0.02,
                              walls=walls)
    assert_parity(*run_both(case, precision, 7), precision)


@pytest.mark.parametrize("precision", [M.F64, M.F32])
def test_tgv2d_1000_steps(precision):
    """Taylor-Green vortex, D2Q9 64x64 periodic, u0 = 0.02, 1000 steps.

    FP64 is held to the 1e-12 bar.  In FP32 each step rounds at ~10 ulp of |u|
    and the field decays 25-fold over the run, so the error relative to the
    final field is larger: it is held to 5e-5 (relative L2, measured 2.2e-5),
    i.e. ~1e-6 of the initial field; the decay factor itself to 1e-5."""
    case = inputs.tgv2d(64, 0.02)
    r_g, u_g, r_o, u_o = run_both(case, precision, 1000)
    if precision == M.F64:
        assert_parity(r_g, u_g, r_o, u_o, precision)
    else:
        assert np.abs(r_g - r_o).max() <= TOL_R[precision]
        assert rel_l2(u_g, u_o) <= 5e-5
    k = 2 * math.pi / 64
    amp = np.sum(u_g * case.u) / np.sum(case.u * case.u)
    assert amp == pytest.approx(((1 + 2 * math.cos(k)) / 3) ** 1000, rel=1e-5)


def test_physical_units_roundtrip():
    """Couette set-up of Test 1 in SI units (dx = 0.02, nu = 0.001): the library's
    unit map (e = 6 nu / dx) must agree with the oracle's."""
    dx, nu = 0.02, 0.001
    e, dt = orc.params(dx, nu)
    case = inputs.channel2d(20, 51, u_top=0.1 / e)
    s = M.Solver(M.D2Q9, case.dims, dx, nu, M.F64, case.periodic, case.node_type, case.wall_rho,
                 np.asarray(case.wall_u) * e)
    p = s.params
    assert p["e"] == pytest.approx(e, rel=1e-15) and p["dt"] == pytest.approx(dt, rel=1e-15)
    g = inputs.rng(40)
    rho = 1 + 0.01 * g.uniform(-1, 1, size=case.grid)
    u = 0.02 * g.uniform(-1, 1, size=(2,) + case.grid)
    s.set_state(rho, u)
    s.step(5)
    r_g, u_g = s.get_state()
    # the same start in lattice units (rho0 = 1): walls take their lattice values
    rl, ul = inputs.place_walls(rho, u / e, case.node_type, case.wall_rho, case.wall_u)
    rl, ul = orc.step(D2, rl, ul, case.periodic, wall=case.wall_mask, nsteps=5)
    r_o, u_o = orc.to_physical(rl, ul, dx, nu)
    assert np.abs(r_g - r_o).max() < 1e-13
    assert np.abs(u_g - u_o).max() < 1e-13 * e


@pytest.mark.parametrize("lat,dims,periodic,walls", [
    (D2, (1, 1), 0b11, "none"), (D3, (1, 1, 1), 0b111, "none"), (D2, (2, 2), 0b11, "none"),
    (D2, (3, 3), 0b00, "box"), (D3, (3, 3, 3), 0b000, "box"), (D2, (2, 5), 0b00, "box"),
    (D3, (1, 4, 3), 0b001, "box")])
def test_degenerate_sizes(lat, dims, periodic, walls):
    case = inputs.random_case(lat, dims, periodic, seed=33, u_amp=0.05, walls=walls)
    assert_parity(*run_both(case, M.F64, 3), M.F64)


def test_zero_steps_and_resume_bit_identical():
    case = inputs.random_case(D3, (12, 11, 10), 0b011, seed=34, walls="box")
    s = M.Solver.from_case(case, M.F32)
    s.step(0)
    r0, u0 = s.get_state()
    assert np.abs(u0 - case.u).max() < 1e-7
    s.step(4)
    snap = s.get_lattice_state()
    s.step(5)
    ref = s.get_lattice_state().copy()
    s.set_lattice_state(snap)
    s.step(5)
    assert np.array_equal(s.get_lattice_state(), ref)
    s.close()


def test_device_pointers_through_torch():
    torch = pytest.importorskip("torch")
    case = inputs.random_case(D2, (64, 48), 0b11, seed=35)
    s = M.Solver(D2, case.dims, 1.0, 1 / 6, M.F32, case.periodic)
    rho = torch.tensor(case.rho, dtype=torch.float32, device="cuda")
    u = torch.tensor(case.u, dtype=torch.float32, device="cuda")
    s.set_state(rho, u)
    s.step(3)
    r2 = torch.empty_like(rho)
    u2 = torch.empty_like(u)
    s.get_state_into(r2, u2)
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, nsteps=3)
    assert rel_l2(u2.double().cpu().numpy(), u_o) < 1e-5
    s.close()


@pytest.mark.parametrize("lat,n", [(D3, 128), (D2, 1024)])
def test_full_size_box_walls(lat, n):
    """At the benchmark sizes (128^3 D3Q19, 1024^2 D2Q9), FP32, in the launch
    configuration the benchmark uses: whole fields against the oracle."""
    dims = (n,) * (3 if lat == D3 else 2)
    case = inputs.random_case(lat, dims, 0, seed=36, u_amp=0.08, rho_amp=0.02, walls="box")
    assert_parity(*run_both(case, M.F32, 3), M.F32)


@pytest.mark.parametrize("lo,hi", [(0.5, 2.0), (30.0, 42.0), (1e-3, 1e3)])
def test_pair_reciprocal_error_bound(lo, hi):
    """The FP32 kernels divide by 1 + drho' and 36 + R through a hardware
    reciprocal refined by one Newton-Raphson step: within one ulp (2^-23
    relative) of 1/x over the ranges those arguments take, and beyond."""
    err = M.maclab_check_reciprocal(lo, hi, 1 << 20)
    assert 0.0 <= err <= 2.0 ** -23


def test_fp32_peak_measurement():
    """The device's paired-FP32 FMA rate: a GB300 (152 SMs x 128 lanes x 2 flops
    at about 2 GHz) gives some tens of TFLOP/s."""
    t = M.maclab_measure_fp32_peak()
    assert 20.0 < t < 250.0
