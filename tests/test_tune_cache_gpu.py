"""MACLAB_TUNE_CACHE: the tuner appends each shape it tunes to the named file
and takes a shape found there instead of timing candidates."""

import pytest

from paper_1901_02716_gb300 import inputs
from paper_1901_02716_gb300 import maclab as M

pytestmark = pytest.mark.gpu


def _lines(path):
    return [ln.split() for ln in path.read_text().splitlines() if ln.strip()] if path.exists() else []


def test_tune_cache_file_is_written_and_read(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("MACLAB_TUNE_CACHE", str(path))
    # shapes no other test tunes (the in-process cache would answer first)
    case1 = inputs.random_case(M.D3Q19, (48, 24, 21), 0b000, seed=71, walls="box")
    s = M.Solver.from_case(case1, M.F32)
    s.tune()
    s.close()
    lines = _lines(path)
    assert len(lines) == 1
    key1, kern1 = lines[0][0], int(lines[0][1])
    assert len(lines[0]) == 5 and lines[0][4] in ("0", "1")  # the launch overlap chosen
    fields = key1.split("/")
    assert fields[2:5] == ["48", "24", "21"]
    assert kern1 in (M.KERNEL_TILED, M.KERNEL_FOLDED)

    # plant a choice for another shape: the tuner adopts it without timing
    fields[4] = "23"
    key2 = "/".join(fields)
    with path.open("a") as f:
        f.write(f"{key2} {M.KERNEL_TILED} 8 5 0\n")
    case2 = inputs.random_case(M.D3Q19, (48, 24, 23), 0b000, seed=72, walls="box")
    t = M.Solver.from_case(case2, M.F32)
    assert t.launch_overlap() == 1
    assert t.tune() == (8, 5)
    assert t.kernel_info()["kernel"] == M.KERNEL_TILED
    assert t.launch_overlap() == 0
    t.step(3)  # the adopted shape runs
    t.close()
    assert len(_lines(path)) == 2  # nothing appended for a shape found in the file


def test_tune_cache_ignores_malformed_lines(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    path.write_text("garbage\n1 2\n")
    monkeypatch.setenv("MACLAB_TUNE_CACHE", str(path))
    case = inputs.random_case(M.D3Q19, (48, 24, 25), 0b000, seed=73, walls="box")
    s = M.Solver.from_case(case, M.F32)
    s.tune()
    s.step(2)
    s.close()
    assert len(_lines(path)) == 3
