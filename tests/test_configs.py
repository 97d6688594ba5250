"""The workload configs: JSON round trip, validation, and the cases they build."""

import itertools
import json

import numpy as np
import pytest

from paper_1901_02716_gb300 import configs, inputs


def test_round_trip():
    text = configs.dumps(configs.WORKLOADS)
    assert configs.loads(text) == configs.WORKLOADS
    one = json.dumps(json.loads(text)[0])
    assert configs.loads(one) == [configs.WORKLOADS[0]]


def test_file_load(tmp_path):
    p = tmp_path / "w.json"
    p.write_text(configs.dumps(configs.WORKLOADS[:2]))
    assert configs.load(str(p)) == configs.WORKLOADS[:2]


@pytest.mark.parametrize("bad", [
    {"name": "x", "kind": "poiseuille", "sides": [8], "precisions": ["f32"], "steps": 1},
    {"name": "x", "kind": "tgv2d", "sides": [8], "precisions": ["f8"], "steps": 1},
    {"name": "x", "kind": "cavity2d", "sides": [8], "precisions": ["f32"], "steps": 1},
    {"name": "x", "kind": "tgv2d", "sides": [], "precisions": ["f32"], "steps": 1},
    {"name": "x", "kind": "batch_cavity2d", "sides": [], "precisions": ["f32"], "steps": 1},
    {"name": "x", "kind": "tgv2d", "sides": [8], "precisions": ["f32"], "steps": 1, "lid": 0.1},
])
def test_rejects_bad_workloads(bad):
    with pytest.raises(ValueError):
        configs.loads(json.dumps(bad))


def test_cases_follow_the_inputs_module():
    tgv = next(configs.WORKLOADS[0].cases())
    assert tgv[0] == "tgv2d/64/f64" and tgv[2] == "f64"
    ref = inputs.tgv2d(64, 0.02)
    assert np.array_equal(tgv[1].u, ref.u) and tgv[1].periodic == 0b11

    cav = list(itertools.islice(configs.WORKLOADS[1].cases(), 2))
    assert [c[0] for c in cav] == ["cavity2d/256/re100/f32", "cavity2d/256/re1000/f32"]
    lid = cav[1][1].wall_u[1, 0]
    assert lid == pytest.approx(inputs.lid_speed(1000.0, 256))

    small_batch = configs.Workload("b", "batch_cavity2d", sides=[], precisions=["f32"], steps=10,
                                   count=3, seed=4)
    label, cases, prec = next(small_batch.cases())
    sides, _, lids = inputs.batch_cavity_sides(3, 4)
    assert label == "b/3/f32" and [c.dims[0] for c in cases] == sides
    assert [c.wall_u[1, 0] for c in cases] == pytest.approx(lids)

    n_cases = sum(1 for w in configs.WORKLOADS if w.kind != "batch_cavity2d"
                  for _ in itertools.product(w.precisions, w.sides, w.re or [None]))
    assert n_cases == 1 + 8 + 4 + 1
