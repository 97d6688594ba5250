"""The C-ABI library loads, exports every declared symbol and validates its input.

CPU-only: no call here reaches a kernel.  maclab_create's argument checks run
before any device allocation, so they can be exercised without a GPU.
"""
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from paper_1901_02716_gb300 import _build, inputs
from paper_1901_02716_gb300 import maclab as M


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return M.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(maclab_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "maclab_step" in names and "maclab_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", M.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(maclab_\w+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in names:
        assert hasattr(lib, n)
    # the binding covers every declared call
    assert set(names) <= set(M.SIGNATURES)


def test_status_strings(lib):
    for s in (M.OK, M.WARN_RLE, M.ERR_INVALID, M.ERR_CUDA, M.ERR_NONFINITE, M.ERR_TIMEOUT,
              M.ERR_OOM, M.ERR_UNSUPPORTED):
        assert M.maclab_status_string(s).startswith("MACLAB_")
    assert "unknown" in M.maclab_status_string(1234)
    assert "sm_103a" in M.maclab_version()


def _create_err(**kw):
    base = dict(lattice=M.D2Q9, dims=(8, 8), dx=1.0, nu=1 / 6, periodic=3)
    base.update(kw)
    with pytest.raises(M.MacLABError) as ei:
        M.Solver(**base)
    return ei.value.status


def test_create_validates_arguments(lib):
    assert _create_err(dx=0.0) == M.ERR_INVALID
    assert _create_err(nu=-1.0) == M.ERR_INVALID
    assert _create_err(dims=(8, 8, 2)) == M.ERR_INVALID          # D2Q9 with nz != 1
    assert _create_err(dims=(0, 8)) == M.ERR_INVALID
    assert _create_err(lattice=7) == M.ERR_INVALID
    assert _create_err(precision=9) == M.ERR_INVALID
    assert _create_err(periodic=1) == M.ERR_INVALID              # y closed, no walls
    # fluid node on a closed boundary
    nt = np.zeros((8, 8), dtype=np.uint8)
    nt[0, :] = 1
    assert _create_err(periodic=1, node_type=nt, wall_u=[[0, 0]]) == M.ERR_INVALID
    # wall id beyond the table
    case = inputs.cavity2d(8)
    assert _create_err(periodic=0, node_type=case.node_type, wall_u=[[0, 0]]) == M.ERR_INVALID


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(M, "_lib", None)
    monkeypatch.setattr(M, "library_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(M.MacLABError):
        M.lib()


def test_noalloc_diagnostics_refuses_host_buffers(lib):
    """maclab_diagnostics_noalloc checks that its buffers are device memory
    before it launches anything: host arrays give MACLAB_ERR_INVALID (here
    without a GPU, where no pointer can be device memory) and stay untouched."""
    state = np.zeros(4 * 64, dtype=np.float32)
    out = np.full(9, 3.0)
    with pytest.raises(M.MacLABError) as ei:
        M.maclab_diagnostics_noalloc(M.D3Q19, M.F32, 64, state.ctypes.data, None, None,
                                     out.ctypes.data, None)
    assert ei.value.status == M.ERR_INVALID
    assert np.all(out == 3.0)


def test_debug_bounds_unsupported_in_normal_build(lib):
    """maclab_debug_bounds exists only in the bounds-checked debug build."""
    with pytest.raises(M.MacLABError) as ei:
        M.maclab_debug_bounds()
    assert ei.value.status == M.ERR_UNSUPPORTED
