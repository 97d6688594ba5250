"""The allocation-free diagnostics entry point against the handle's diagnostics.

maclab_diagnostics_noalloc serves callers that cannot allocate device memory
while they run (a host loop that has reserved all device memory for its own
pool, or code that may not block on an allocation): its scratch is a fixed
array the library reserves at load time.  Here it is called through the C ABI
on a state read back from a handle, twice in a row, and its sums must give the
same diagnostics as maclab_diagnostics on that handle.  This file is collected
last so that a failing run has already run every other test; it passes both on
its own in a fresh process and after the rest of the suite.
"""
import math

import numpy as np
import pytest

from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_02716_gb300 import _build
    _build.build()


def storage_order(case):
    """Node types in the library's storage order (the two halves of each x row
    interleaved when nx is a multiple of 4, as maclab.h documents)."""
    nt = case.node_type.reshape(-1, case.dims[0])
    nx = case.dims[0]
    if nx % 4:
        return nt.reshape(-1).copy()
    h = nx // 2
    pos = np.array([2 * (x % h) + (x >= h) for x in range(nx)])
    out = np.empty_like(nt)
    out[:, pos] = nt
    return out.reshape(-1).copy()


@pytest.mark.parametrize("lat,dims,periodic,walls", [
    (inputs.D3Q19, (32, 20, 12), 0b000, "box"),      # interleaved rows, walls excluded
    (inputs.D2Q9, (30, 17), 0b01, "mixed"),          # plain order, mask walls
    (inputs.D2Q9, (64, 48), 0b11, "none"),           # no walls
])
def test_noalloc_matches_handle_diagnostics(lat, dims, periodic, walls):
    torch = pytest.importorskip("torch")
    case = inputs.random_case(lat, dims, periodic, seed=61, u_amp=0.08, rho_amp=0.02,
                              walls=walls)
    s = M.Solver.from_case(case, M.F32)          # dx = 1, nu = 1/6: e = 1, rho0 = 1
    nbytes = s.state_bytes()
    prev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    cur = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s.step(4)
    s.get_lattice_state(prev)
    s.step(1)
    s.get_lattice_state(cur)
    ref = s.diagnostics()                        # the existing entry point
    n_fluid = s.params["n_fluid"]
    s.close()

    excl = None
    if case.node_type is not None:
        excl = torch.from_numpy((storage_order(case) != 0).astype(np.uint8)).cuda()
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream or None
    n = case.n_nodes
    results = []
    for _ in range(2):                           # two calls in a row share the scratch
        out.fill_(float("nan"))
        M.maclab_diagnostics_noalloc(lat, M.F32, n, cur.data_ptr(), prev.data_ptr(),
                                     None if excl is None else excl.data_ptr(),
                                     out.data_ptr(), stream)
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    for sums in results:
        assert np.all(np.isfinite(sums))
        assert n_fluid + sums[0] == pytest.approx(ref["mass"], rel=1e-12)
        assert 0.5 * sums[1] == pytest.approx(ref["kinetic"], rel=1e-12)
        for i in range(len(dims)):
            assert sums[2 + i] == pytest.approx(ref["momentum"][i], rel=1e-10, abs=1e-12)
        assert math.sqrt(sums[5] / sums[6]) == pytest.approx(ref["residual"], rel=1e-12)
        assert sums[7] == pytest.approx(ref["max_u_lattice"], rel=1e-15)
        assert sums[8] == ref["nonfinite"] == 0
    assert np.array_equal(results[0], results[1])


def test_noalloc_rejects_oversized_input():
    with pytest.raises(M.MacLABError) as ei:
        M.maclab_diagnostics_noalloc(inputs.D3Q19, M.F32, 33554432 + 1, 1, None, None, 1)
    assert ei.value.status == M.ERR_INVALID
    assert "33554432" in str(ei.value)
