"""Host buffers that are page-locked are read and written by the conversion
kernels directly; the state they give and receive must be the same bits as
through pageable memory and the staging buffer."""

import numpy as np
import pytest

from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu


def _pinned(a):
    torch = pytest.importorskip("torch")
    t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0].copy()).dtype).pin_memory()
    t.numpy()[...] = a
    return t


@pytest.mark.parametrize("lat,dims,periodic,walls", [(M.D3Q19, (32, 16, 12), 0b000, "box"),
                                                     (M.D2Q9, (64, 37), 0b01, "mixed")])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_pinned_host_buffers_match_pageable(lat, dims, periodic, walls, dtype):
    case = inputs.random_case(lat, dims, periodic, seed=81, u_amp=0.06, rho_amp=0.02, walls=walls)
    rho = case.rho.astype(dtype)
    u = case.u.astype(dtype)
    t_rho, t_u = _pinned(rho), _pinned(u)        # keep the tensors alive
    out = []
    for pinned in (False, True):
        s = M.Solver.from_case(case, M.F32)
        if pinned:
            s.set_state(t_rho.numpy(), t_u.numpy())
        else:
            s.set_state(rho, u)
        first = s.get_lattice_state().copy()
        s.step(5)
        if pinned:
            g_rho, g_u = _pinned(np.zeros_like(rho)), _pinned(np.zeros_like(u))
            s.get_state_into(g_rho.numpy(), g_u.numpy())
            got = (g_rho.numpy().copy(), g_u.numpy().copy())
        else:
            got = (np.zeros_like(rho), np.zeros_like(u))
            s.get_state_into(*got)
        out.append((first, s.get_lattice_state().copy(), got))
        s.close()
    (a0, a1, ag), (b0, b1, bg) = out
    assert np.array_equal(a0, b0)
    assert np.array_equal(a1, b1)
    assert np.array_equal(ag[0], bg[0]) and np.array_equal(ag[1], bg[1])
