"""The bounds-checked debug build of the library (MACLAB_BOUNDS_CHECK).

The debug build's D3Q19 two-rows-per-thread kernel compares every global and
shared-memory index with the size of its buffer and records (and skips) any
access outside it.  Over the kernel's awkward shapes -- rows narrower than the
block (idle lanes), one quad per row (both x-walls in one lane), every
periodicity, obstacle masks, 4- and 8-row tiles, 16-bit storage -- it must
record nothing, and give results bitwise equal to the normal build's (the
checks only guard accesses).  The debug library runs in a subprocess.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu

CASES = [
    ((128, 16, 11), 0b000, "box", 8, "f32"),
    ((96, 12, 10), 0b010, "mixed", 4, "f32"),
    ((124, 8, 5), 0b001, "box", 0, "f32"),
    ((60, 16, 7), 0b111, "none", 0, "f32"),
    ((4, 8, 6), 0b000, "box", 0, "f32"),
    ((8, 16, 7), 0b010, "box", 0, "f32"),
    ((64, 24, 13), 0b110, "mixed", 8, "bf16"),
]

SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1901_02716_gb300 import inputs, maclab as M
out = sys.argv[2]
cases = eval(sys.argv[3])
res = {}
for i, (dims, per, walls, ty, prec) in enumerate(cases):
    case = inputs.random_case(inputs.D3Q19, dims, per, seed=91, u_amp=0.08, rho_amp=0.02, walls=walls,
                              force=(1e-4, -2e-4, 3e-4))
    s = M.Solver.from_case(case, {"f32": M.F32, "bf16": M.BF16_STORE}[prec])
    s.set_kernel(M.KERNEL_ROWS2)
    if ty:
        s.set_tile(ty, 0)
    s.step(3)
    r, u = s.get_state()
    s.close()
    res[f"r{i}"], res[f"u{i}"] = r, u
count, first = M.maclab_debug_bounds()
res["count"], res["first"] = np.array(count), np.array(first)
np.savez(out, **res)
"""


def test_checked_build_records_nothing_and_matches(tmp_path):
    from paper_1901_02716_gb300 import _build
    _build.build()
    lib = _build.build(bounds_check=True)
    out = str(tmp_path / "checked.npz")
    env = dict(os.environ, MACLAB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, out, repr(CASES)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(out)
    assert int(got["count"]) == 0, f"first bad index {int(got['first'])}"
    for i, (dims, per, walls, ty, prec) in enumerate(CASES):
        case = inputs.random_case(inputs.D3Q19, dims, per, seed=91, u_amp=0.08, rho_amp=0.02, walls=walls,
                                  force=(1e-4, -2e-4, 3e-4))
        s = M.Solver.from_case(case, {"f32": M.F32, "bf16": M.BF16_STORE}[prec])
        s.set_kernel(M.KERNEL_ROWS2)
        if ty:
            s.set_tile(ty, 0)
        s.step(3)
        rr, uu = s.get_state()
        s.close()
        assert np.array_equal(rr, got[f"r{i}"]) and np.array_equal(uu, got[f"u{i}"]), dims
