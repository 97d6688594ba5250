"""GPU parity of the D3Q19 kernel with two rows per thread (MACLAB_KERNEL_ROWS2)
against the FP64 CPU oracle, element by element on the same seeded inputs.

Cases span the kernel's shapes (16- and 32-quad rows, tiles of 4 and 8 rows), rows narrower than the block (idle lanes), every periodicity, box walls
with the x-wall lanes (one quad per row: both x-walls in one lane; two lanes
with one x-wall each), random obstacle masks, and a body force.  Bars as in
test_parity_gpu.py: FP32 <= 1e-5 relative L2 on u and <= 1e-6 absolute on rho;
16-bit storage within its stated storage error.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M
from test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu

D3 = inputs.D3Q19


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


ROWS2_CASES = [
    ((8, 8, 5), 0b111, "none", 0),
    ((12, 8, 9), 0b000, "box", 0),
    ((16, 16, 19), 0b101, "mixed", 0),
    ((32, 16, 7), 0b011, "box", 0),
    ((128, 8, 6), 0b000, "box", 0),
    ((96, 12, 10), 0b010, "mixed", 0),     # 24 of 32 lanes, tile of 4 rows
    ((4, 8, 3), 0b111, "none", 0),
    ((20, 16, 17), 0b100, "mixed", 0),
    ((128, 4, 9), 0b111, "none", 0),
    ((128, 16, 11), 0b000, "box", 8),
    ((128, 12, 10), 0b000, "box", 4),
    ((64, 24, 13), 0b110, "mixed", 8),
    ((64, 32, 9), 0b010, "box", 0),
    ((124, 8, 5), 0b001, "box", 0),        # 31 of 32 lanes, periodic x
    ((60, 16, 7), 0b000, "box", 0),        # 15 of 16 lanes
    ((4, 8, 6), 0b000, "box", 0),          # one quad per row: both x-walls in one lane
    ((8, 16, 7), 0b010, "box", 0),         # two lanes, one x-wall each
]


KERNELS = [M.KERNEL_ROWS2]


def _supported(kernel, dims, ty):
    return ty in (0, 4, 8)


def _run(case, precision, steps, ty=0, kernel=M.KERNEL_ROWS2):
    s = M.Solver.from_case(case, precision)
    s.set_kernel(kernel)
    if ty:
        s.set_tile(ty, 0)
    assert s.kernel_info()["kernel"] == kernel
    s.step(steps)
    s.sync()  # raises if a bounded wait for a tile copy ran out (MACLAB_ERR_TIMEOUT)
    out = s.get_state()
    s.close()
    return out


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("dims,periodic,walls,ty", ROWS2_CASES)
@pytest.mark.parametrize("steps", [1, 5])
def test_rows2_kernel(kernel, dims, periodic, walls, ty, steps):
    if not _supported(kernel, dims, ty):
        pytest.skip("tile shape not built for this kernel")
    case = inputs.random_case(D3, dims, periodic, seed=43, u_amp=0.08, rho_amp=0.02,
                              walls=walls, force=(1e-4, -2e-4, 3e-4))
    r_g, u_g = _run(case, M.F32, steps, ty, kernel)
    r_o, u_o = orc.step(D3, case.rho, case.u, case.periodic, wall=case.wall_mask,
                        force=case.force, nsteps=steps)
    assert_parity(r_g, u_g, r_o, u_o, M.F32)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("dims,periodic,walls,ty", ROWS2_CASES)
def test_rows2_matches_tiled_kernel(kernel, dims, periodic, walls, ty):
    """Other terms and order than the tiled kernel: FP32 results agree to rounding."""
    if not _supported(kernel, dims, ty):
        pytest.skip("tile shape not built for this kernel")
    case = inputs.random_case(D3, dims, periodic, seed=44, u_amp=0.08, rho_amp=0.02, walls=walls)
    r1, u1 = _run(case, M.F32, 10, 0, M.KERNEL_TILED)
    r2, u2 = _run(case, M.F32, 10, ty, kernel)
    assert np.abs(r1 - r2).max() < 1e-6
    assert np.abs(u1 - u2).max() < 2e-6 * np.abs(u1).max()


@pytest.mark.parametrize("kernel", KERNELS)
def test_rows2_walls_unchanged_and_state_finite(kernel):
    """Wall nodes keep their values exactly (they are never computed into)."""
    case = inputs.random_case(D3, (32, 16, 12), 0b000, seed=45, u_amp=0.08, rho_amp=0.02,
                              walls="box")
    r, u = _run(case, M.F32, 9, 0, kernel)
    w = case.wall_mask.astype(bool)
    assert np.array_equal(r[w].astype(np.float32), case.rho[w].astype(np.float32))
    assert np.array_equal(u[:, w].astype(np.float32), case.u[:, w].astype(np.float32))
    assert np.isfinite(r).all() and np.isfinite(u).all()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", [M.BF16_STORE, M.F16_STORE])
@pytest.mark.parametrize("dims,periodic,walls,ty", [((128, 8, 6), 0b000, "box", 0),
                                                    ((96, 16, 10), 0b010, "mixed", 0),
                                                    ((128, 16, 11), 0b000, "box", 8),
                                                    ((64, 8, 5), 0b111, "none", 0)])
def test_rows2_kernel_16bit_storage(kernel, precision, dims, periodic, walls, ty):
    case = inputs.random_case(D3, dims, periodic, seed=46, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=(1e-4, -2e-4, 3e-4))
    r_g, u_g = _run(case, precision, 7, ty, kernel)
    r_o, u_o = orc.step(D3, case.rho, case.u, case.periodic, wall=case.wall_mask, force=case.force,
                        nsteps=7)
    assert_parity(r_g, u_g, r_o, u_o, precision)
