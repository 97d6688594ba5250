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


def _cases():
    small = [
        # (label, case builder, storage type)
        ("d3q19-box-f32", lambda: inputs.random_case(inputs.D3Q19, (32, 20, 12), 0b000, seed=61,
                                                     u_amp=0.08, rho_amp=0.02, walls="box"), M.F32),
        ("d3q19-box-f64", lambda: inputs.random_case(inputs.D3Q19, (32, 20, 12), 0b000, seed=62,
                                                     u_amp=0.08, rho_amp=0.02, walls="box"), M.F64),
        ("d3q19-box-bf16", lambda: inputs.random_case(inputs.D3Q19, (32, 20, 12), 0b000, seed=63,
                                                      u_amp=0.08, rho_amp=0.02, walls="box"),
         M.BF16_STORE),
        ("d2q9-mask-f32", lambda: inputs.random_case(inputs.D2Q9, (30, 17), 0b01, seed=64,
                                                     u_amp=0.08, rho_amp=0.02, walls="mixed"), M.F32),
        ("d2q9-periodic-f32", lambda: inputs.random_case(inputs.D2Q9, (64, 48), 0b11, seed=65,
                                                         u_amp=0.08, rho_amp=0.02), M.F32),
    ]
    large = [
        # 2,097,152 nodes: 256 partial blocks
        ("cavity3d-128-f32", lambda: inputs.cavity3d(128, lid=inputs.lid_speed(100.0, 128)), M.F32),
        # 33,524,100 nodes: 4093 of the 4096 partial blocks the fixed array holds
        ("cavity2d-5790-f32", lambda: inputs.cavity2d(5790, lid=inputs.lid_speed(1000.0, 5790)),
         M.F32),
    ]
    return small + large


@pytest.mark.parametrize("label,make,precision", _cases(), ids=[c[0] for c in _cases()])
def test_noalloc_matches_handle_diagnostics(label, make, precision):
    torch = pytest.importorskip("torch")
    case = make()
    lat = case.lattice
    s = M.Solver.from_case(case, precision)      # dx = 1, nu = 1/6: e = 1, rho0 = 1
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
        M.maclab_diagnostics_noalloc(lat, precision, n, cur.data_ptr(), prev.data_ptr(),
                                     None if excl is None else excl.data_ptr(),
                                     out.data_ptr(), stream)
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    # The stored density deviations are summed node by node on both paths
    # (float-float, or FP64): mass agrees to 1e-12.  The per-node products
    # (rho |u|^2, rho u_i, the residual's squares) are rounded to the arithmetic
    # type on both paths, but the handle's row kernel adds a quad's four in that
    # type before its float-float sum, and fuses the product into that add: with
    # FP32 arithmetic (FP32 and 16-bit storage) each term differs by at most 5
    # units of 2^-24 of its magnitude, so the sums differ by at most
    # 5 * 2^-24 * sum |term|; with FP64 storage the same count of 2^-53 units.
    rel = 5 * 2.0 ** -24 if precision != M.F64 else 1e-12
    # momentum sums cancel: their rounding is bounded by the sum of |rho u_i|,
    # at most n (1 + max |drho|) |u|max, not by the sum itself
    mom_abs = max(rel, 1e-12) * n * 1.1 * max(ref["max_u_lattice"], 1e-30)
    for sums in results:
        assert np.all(np.isfinite(sums))
        assert n_fluid + sums[0] == pytest.approx(ref["mass"], rel=1e-12)
        assert 0.5 * sums[1] == pytest.approx(ref["kinetic"], rel=rel)
        for i in range(case.d):
            assert sums[2 + i] == pytest.approx(ref["momentum"][i], rel=1e-10, abs=mom_abs)
        # the residual's ratio: each of its two sums within rel
        assert math.sqrt(sums[5] / sums[6]) == pytest.approx(ref["residual"], rel=rel)
        assert sums[7] == pytest.approx(ref["max_u_lattice"], rel=1e-15)
        assert sums[8] == ref["nonfinite"] == 0
    assert np.array_equal(results[0], results[1])


def test_noalloc_rejects_oversized_input():
    with pytest.raises(M.MacLABError) as ei:
        M.maclab_diagnostics_noalloc(inputs.D3Q19, M.F32, 33554432 + 1, 1, None, None, 1)
    assert ei.value.status == M.ERR_INVALID
    assert "33554432" in str(ei.value)


def test_noalloc_rejects_host_buffers():
    """A host out_sums (or state) is refused before any launch; a device
    buffer it would have written stays untouched."""
    torch = pytest.importorskip("torch")
    n = 4096
    state = torch.zeros(4 * n, dtype=torch.float32, device="cuda")
    out_dev = torch.full((9,), 7.0, dtype=torch.float64, device="cuda")
    out_host = np.full(9, 7.0)
    state_host = np.zeros(4 * n, dtype=np.float32)
    for st, o in ((state.data_ptr(), out_host.ctypes.data), (state_host.ctypes.data, out_dev.data_ptr())):
        with pytest.raises(M.MacLABError) as ei:
            M.maclab_diagnostics_noalloc(inputs.D3Q19, M.F32, n, st, None, None, o, None)
        assert ei.value.status == M.ERR_INVALID
    torch.cuda.synchronize()
    assert np.all(out_host == 7.0)
    assert torch.all(out_dev == 7.0)
