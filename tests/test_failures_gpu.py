"""Failure detection without a GPU fault: the lattice Reynolds number warning
of maclab_create, a device allocation the GPU cannot satisfy (refused by the
allocator, nothing is held), and a context that stays usable afterwards."""

import numpy as np
import pytest

from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu


def test_lattice_reynolds_warning():
    # at tau = 1 the lattice Reynolds number of a wall is 6 |u_w| / e: lid 0.2 gives 1.2
    s = M.Solver.from_case(inputs.cavity2d(32, lid=0.2), M.F32)
    assert s.create_status == M.WARN_RLE
    assert s.params["R_le"] == pytest.approx(1.2)
    s.step(3)                       # a warning, not an error: the handle steps
    s.close()
    t = M.Solver.from_case(inputs.cavity2d(32, lid=0.1), M.F32)
    assert t.create_status == M.OK
    t.close()


def test_device_allocation_failure_is_reported():
    # 4096^3 nodes in FP64: 2.2 TB per state buffer, refused at the first allocation
    with pytest.raises(M.MacLABError) as ei:
        M.Solver(M.D3Q19, (4096, 4096, 4096), 1.0, 1.0 / 6.0, M.F64, periodic=0b111)
    assert ei.value.status == M.ERR_OOM
    # the context is still usable and a normal domain steps to the same bits
    case = inputs.cavity2d(48, lid=0.05)
    out = []
    for _ in range(2):
        s = M.Solver.from_case(case, M.F32)
        s.step(4)
        out.append(s.get_lattice_state().copy())
        s.close()
    assert np.array_equal(out[0], out[1])
