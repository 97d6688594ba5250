"""Host-side logic of bench.py on the CPU: the reference arm's JSON line, and
the multi-rank path (barrier, max over ranks, rank 0 prints) with gloo ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.strip().startswith("{")]


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--side", "12", "--steps",
                        "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_under_two_gloo_ranks():
    env = dict(os.environ, MACLAB_BENCH_BACKEND="gloo", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2", "--side",
                        "10", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"


def _rank(rank, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank), MACLAB_BENCH_BACKEND="gloo")
    r, w, _ = bench.dist_init()
    bench.dist_barrier(w)
    q.put((r, bench.dist_max(float(10 + 5 * rank), w)))
    dist.destroy_process_group()


def test_dist_max_over_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(i, port, q)) for i in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 15.0), (1, 15.0)]


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    """bench.py reports an ncu traffic figure only while the profiled sources
    are unchanged (same hash), and only for the profiled kernel."""
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.md").write_text(
        "# title\n\nkernel_tag: step_fold<D3Q19,f32>\nsource_sha256: 0123456789abcdef\n"
        "traffic_bytes_per_launch: 12345678\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("step_fold<D3Q19,f32>", "0123456789abcdef") == 12345678.0
    assert bench.traffic_from_profiles("step_fold<D3Q19,f32>", "fedcba9876543210") is None
    assert bench.traffic_from_profiles("segment<D2Q9,f32>", "0123456789abcdef") is None


def test_committed_profiles_are_well_formed():
    """Every ncu summary names the command that made it; those that carry a
    traffic figure give the kernel, a 16-digit source hash and a number."""
    import re
    pdir = os.path.join(ROOT, "profiles")
    names = [n for n in os.listdir(pdir) if n.endswith(".md")]
    assert names
    for n in names:
        txt = open(os.path.join(pdir, n)).read()
        assert "ncu " in txt and "--clock-control none" in txt, n
        if re.search(r"^kernel_tag:", txt, re.M):
            assert re.search(r"^source_sha256:\s*[0-9a-f]{16}\s*$", txt, re.M), n
            assert re.search(r"^traffic_bytes_per_launch:\s*[0-9]+\s*$", txt, re.M), n
