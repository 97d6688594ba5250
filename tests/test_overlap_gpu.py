"""Programmatic dependent launch of the step kernels: with the overlap on (the
default) each step's kernel waits on the device for the previous one, so the
state after any number of steps, in graphs or single launches, must be the
same bits as with plain stream-ordered launches."""

import numpy as np
import pytest

from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu

D2, D3 = M.D2Q9, M.D3Q19

# (lattice, dims, periodic, walls, precision, kernel, (ty, tz))
CASES = [
    (D3, (64, 32, 40), 0b000, "box", M.F32, M.KERNEL_FOLDED, (0, 0)),
    (D3, (48, 24, 17), 0b111, "none", M.F64, M.KERNEL_TILED, (0, 0)),
    (D3, (96, 12, 21), 0b010, "mixed", M.BF16_STORE, M.KERNEL_FOLDED, (0, 0)),
    (D2, (136, 45), 0b01, "mixed", M.F32, M.KERNEL_TILED, (0, 0)),
    (D2, (512, 300), 0b00, "box", M.F32, M.KERNEL_SEGMENT, (0, 4)),
    (D2, (256, 70), 0b10, "box", M.F32, M.KERNEL_SEGMENT, (2, 3)),
    (D2, (96, 41), 0b11, "none", M.F64, M.KERNEL_SEGMENT, (2, 2)),
]


@pytest.mark.parametrize("lat,dims,periodic,walls,prec,kernel,tile", CASES)
def test_overlap_gives_identical_bits(lat, dims, periodic, walls, prec, kernel, tile):
    force = (1e-4, -1e-4, 5e-5) if lat == D3 else (1e-4, -1e-4)
    case = inputs.random_case(lat, dims, periodic, seed=61, u_amp=0.06, rho_amp=0.02, walls=walls,
                              force=force)
    out = []
    for on in (1, 0):
        s = M.Solver.from_case(case, prec)
        s.set_kernel(kernel)
        if tile != (0, 0):
            s.set_tile(*tile)
        s.set_launch_overlap(on)
        s.step(37)   # one 32-step graph and single launches
        s.step(3)
        out.append((s.get_lattice_state(), s.diagnostics()["residual"]))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("depth", [1, 2])
def test_batch_overlap_gives_identical_bits(depth):
    sides = [64, 96, 128, 160, 96, 64]
    cases = [inputs.cavity2d(n, lid=0.05 + 0.01 * i) for i, n in enumerate(sides)]
    states = []
    for on in (1, 0):
        b = M.Batch.from_cases(cases, M.F32)
        b.set_depth(depth)
        b.set_launch_overlap(on)
        b.step(41)
        states.append([m.get_lattice_state() for m in b.members])
        b.close()
    for x, y in zip(*states):
        assert np.array_equal(x, y)


def test_overlap_rejects_bad_values():
    case = inputs.cavity2d(64, lid=0.05)
    s = M.Solver.from_case(case, M.F32)
    with pytest.raises(M.MacLABError):
        s.set_launch_overlap(2)
    s.close()
