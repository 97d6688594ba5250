"""GPU parity of the block-resident D2Q9 kernel (MACLAB_KERNEL_BLOCK): several
steps per launch on tiles held in registers and shared memory.

Every case is compared element by element with the FP64 CPU oracle (the bars
of test_parity_gpu) and bit for bit with the tiled kernel, whose sums run in
the same order.  The cases cover ragged tiles in x and y, rows of one pair
(nx = 4) and of fewer pairs than a tile's halo, the periodic wrap in either
axis (with a tile wrapping the whole domain several times), box walls, mask
walls with interior obstacles, forcing, runs that end in a partial launch,
and the full-size 256^2 and 1024^2 cavities.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu

D2 = inputs.D2Q9
TOL_U = {M.F64: 1e-12, M.F32: 1e-5}
TOL_R = {M.F64: 1e-12, M.F32: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


def rel_l2(a, b):
    nb = np.sqrt(np.sum(b * b))
    return np.sqrt(np.sum((a - b) ** 2)) / (nb if nb > 0 else 1.0)


def assert_oracle(r_g, u_g, r_o, u_o, precision):
    if precision == M.F64:
        assert np.abs(r_g - r_o).max() <= TOL_R[precision] * np.abs(r_o).max()
        assert np.abs(u_g - u_o).max() <= TOL_U[precision] * max(np.abs(u_o).max(), 1e-300)
    else:
        assert np.abs(r_g - r_o).max() <= TOL_R[precision]
        assert rel_l2(u_g, u_o) <= TOL_U[precision]


def run(case, precision, steps, kernel, ty=0):
    s = M.Solver.from_case(case, precision)
    s.set_kernel(kernel)
    if ty:
        s.set_tile(ty, 0)
    s.step(steps)
    s.sync()
    x = s.get_lattice_state().copy()
    r, u = s.get_state()
    res = s.diagnostics()["residual"]
    s.close()
    return x, r, u, res


BLOCK_CASES = [
    # dims, periodic, walls
    ((16, 13), 0b11, "none"),
    ((64, 37), 0b00, "box"),
    ((96, 41), 0b01, "mixed"),
    ((4, 9), 0b11, "none"),     # one pair per half row: the tile wraps the row many times
    ((4, 9), 0b00, "box"),      # both x-walls in one pair
    ((8, 12), 0b10, "box"),
    ((136, 45), 0b01, "mixed"),
    ((248, 70), 0b10, "box"),
    ((200, 3), 0b11, "none"),   # fewer rows than a tile's halo
]


@pytest.mark.parametrize("dims,periodic,walls", BLOCK_CASES)
@pytest.mark.parametrize("precision,ty", [(M.F32, 1), (M.F32, 2), (M.F32, 4), (M.F32, 8),
                                          (M.F64, 1), (M.F64, 2), (M.F64, 4)])
def test_block_kernel(dims, periodic, walls, precision, ty):
    case = inputs.random_case(D2, dims, periodic, seed=51, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=(1e-4, -2e-4))
    steps = 2 * ty + 3  # two full launches, then a partial one and the closing one-step launch
    x, r_g, u_g, res = run(case, precision, steps, M.KERNEL_BLOCK, ty)
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask, force=case.force,
                        nsteps=steps)
    assert_oracle(r_g, u_g, r_o, u_o, precision)
    t, _, _, res_t = run(case, precision, steps, M.KERNEL_TILED)
    assert np.array_equal(x, t)
    assert res == res_t  # the previous state held is step n - 1 in both


@pytest.mark.parametrize("ty", [0, 4, 8])
@pytest.mark.parametrize("steps", [1, 5, 33, 100])
def test_block_runs_and_graphs(ty, steps):
    """Graph-captured runs (32 steps per graph) and the launches after them;
    two calls in a row continue bit-exactly."""
    case = inputs.random_case(D2, (256, 96), 0b00, seed=52, u_amp=0.05, walls="box", force=(1e-4, 0.0))
    s = M.Solver.from_case(case, M.F32)
    s.set_kernel(M.KERNEL_BLOCK)
    s.set_tile(ty, 0)
    info = s.kernel_info()
    assert info["kernel"] == M.KERNEL_BLOCK
    assert info["steps_per_launch"] == (ty or 8)  # default at 12,288 pairs: 8
    s.step(steps)
    s.step(steps + 1)
    s.sync()
    t = M.Solver.from_case(case, M.F32)
    t.set_kernel(M.KERNEL_TILED)
    t.step(2 * steps + 1)
    assert np.array_equal(s.get_lattice_state(), t.get_lattice_state())
    assert s.diagnostics()["residual"] == t.diagnostics()["residual"]
    s.close()
    t.close()


@pytest.mark.parametrize("n", [256, 1024])
def test_block_full_size_cavity(n):
    """The benchmark cavities (box walls, FP32) at full size: 3 steps against
    the oracle over the whole field; 40 steps bit for bit with the tiled kernel."""
    case = inputs.random_case(D2, (n, n), 0, seed=53, u_amp=0.08, rho_amp=0.02, walls="box")
    _, r_g, u_g, _ = run(case, M.F32, 3, M.KERNEL_BLOCK, 4)
    r_o, u_o = orc.step(D2, case.rho, case.u, case.periodic, wall=case.wall_mask, nsteps=3)
    assert_oracle(r_g, u_g, r_o, u_o, M.F32)
    x, _, _, _ = run(case, M.F32, 40, M.KERNEL_BLOCK, 8)
    t, _, _, _ = run(case, M.F32, 40, M.KERNEL_TILED)
    assert np.array_equal(x, t)


def test_block_is_the_small_2d_default():
    """D2Q9 up to 512^2 picks the block kernel (FP32: 8 steps per launch up
    to 65,536 pairs, 4 above; FP64: 4 up to 16,384 pairs, 2 above); larger
    grids keep the segment kernel."""
    for dims, kernel, steps in (((256, 256), M.KERNEL_BLOCK, 8), ((512, 512), M.KERNEL_BLOCK, 4),
                                ((1024, 1024), M.KERNEL_SEGMENT, None)):
        case = inputs.cavity2d(dims[0])
        s = M.Solver.from_case(case, M.F32)
        info = s.kernel_info()
        assert info["kernel"] == kernel
        if steps is not None:
            assert info["steps_per_launch"] == steps
        s.close()
    for n, steps in ((128, 4), (256, 2)):
        s = M.Solver.from_case(inputs.cavity2d(n), M.F64)
        assert s.kernel_info()["kernel"] == M.KERNEL_BLOCK
        assert s.kernel_info()["steps_per_launch"] == steps
        s.close()


def test_block_rejects_unsupported():
    case = inputs.random_case(D2, (64, 16), 0b11, seed=54)
    s = M.Solver.from_case(case, M.F64)
    s.set_kernel(M.KERNEL_BLOCK)
    with pytest.raises(M.MacLABError):
        s.set_tile(8, 0)  # FP64 tiles leave no output rows at 8 steps
    with pytest.raises(M.MacLABError):
        s.set_tile(3, 0)
    s.close()
    s = M.Solver.from_case(case, M.BF16_STORE)
    with pytest.raises(M.MacLABError):
        s.set_kernel(M.KERNEL_BLOCK)
    s.close()
    c3 = inputs.random_case(inputs.D3Q19, (8, 8, 8), 0b111, seed=55)
    s = M.Solver.from_case(c3, M.F32)
    with pytest.raises(M.MacLABError):
        s.set_kernel(M.KERNEL_BLOCK)
    s.close()
