"""The workloads as data: a dataclass per workload, a JSON loader and writer,
and the five flows of the paper's tests as measured here (Taylor-Green vortex,
Test 4; lid-driven cavities, Tests 3 and 5; a batch of cavities; the 3D
Taylor-Green rollout used for gradients).

``Workload.cases()`` builds the seeded synthetic inputs with ``inputs``; it
holds no arithmetic of the method.  Velocities are in lattice units, so a
cavity's Reynolds number sets its lid speed through ``inputs.lid_speed``
(the lattice viscosity is 1/6 at tau = 1).

    from paper_1901_02716_gb300 import configs
    for w in configs.load("workloads.json"):          # or configs.WORKLOADS
        for label, case, precision in w.cases():
            ...
"""
from __future__ import annotations

import dataclasses
import json
from typing import Iterator

from . import inputs

KINDS = ("tgv2d", "cavity2d", "cavity3d", "batch_cavity2d", "tgv3d")
PRECISIONS = ("f64", "f32", "bf16", "f16")


@dataclasses.dataclass
class Workload:
    name: str
    kind: str                      # one of KINDS
    sides: list                    # nodes per side (one case per side; batches: unused)
    precisions: list               # storage types, names of PRECISIONS
    steps: int                     # time steps of a run
    re: list = dataclasses.field(default_factory=list)  # cavities: Reynolds numbers
    u0: float = 0.02               # Taylor-Green amplitude (lattice units)
    noise_sigma: float = 0.0       # tgv3d: seeded Gaussian perturbation of u
    count: int = 0                 # batches: number of domains
    seed: int = 0                  # offset of the base seed of ``inputs``

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"unknown workload kind {self.kind!r}")
        bad = [p for p in self.precisions if p not in PRECISIONS]
        if bad:
            raise ValueError(f"unknown precision(s) {bad}")
        if self.steps < 0:
            raise ValueError("steps must be >= 0")
        if self.kind == "batch_cavity2d":
            if self.count < 1:
                raise ValueError("a batch needs count >= 1")
        elif not self.sides or min(self.sides) < 4:
            raise ValueError("sides must be given, each >= 4")
        if self.kind in ("cavity2d", "cavity3d") and not self.re:
            raise ValueError("cavities need at least one Reynolds number")

    def cases(self) -> Iterator[tuple]:
        """(label, case or list of cases, precision name) for every combination."""
        for prec in self.precisions:
            if self.kind == "tgv2d":
                for n in self.sides:
                    yield f"{self.name}/{n}/{prec}", inputs.tgv2d(n, self.u0), prec
            elif self.kind == "tgv3d":
                for n in self.sides:
                    yield (f"{self.name}/{n}/{prec}",
                           inputs.tgv3d(n, self.u0, self.noise_sigma, self.seed), prec)
            elif self.kind == "cavity2d":
                for n in self.sides:
                    for re in self.re:
                        yield (f"{self.name}/{n}/re{re:g}/{prec}",
                               inputs.cavity2d(n, lid=inputs.lid_speed(re, n)), prec)
            elif self.kind == "cavity3d":
                for n in self.sides:
                    for re in self.re:
                        yield (f"{self.name}/{n}/re{re:g}/{prec}",
                               inputs.cavity3d(n, lid=inputs.lid_speed(re, n)), prec)
            else:
                sides, _, lids = inputs.batch_cavity_sides(self.count, self.seed)
                yield (f"{self.name}/{self.count}/{prec}",
                       [inputs.cavity2d(n, lid=v) for n, v in zip(sides, lids)], prec)


WORKLOADS = [
    Workload("tgv2d", "tgv2d", sides=[64], precisions=["f64"], steps=1000, u0=0.02),
    Workload("cavity2d", "cavity2d", sides=[256, 1024], precisions=["f32", "f64"], steps=20000,
             re=[100.0, 1000.0]),
    Workload("cavity3d", "cavity3d", sides=[128], precisions=["f32", "bf16"], steps=10000,
             re=[100.0, 400.0]),
    Workload("batch_cavities", "batch_cavity2d", sides=[], precisions=["f32"], steps=5000,
             count=64, seed=4),
    Workload("tgv3d_gradient", "tgv3d", sides=[96], precisions=["f32"], steps=2000, u0=0.02,
             noise_sigma=1e-3, seed=5),
]


def dumps(workloads) -> str:
    return json.dumps([dataclasses.asdict(w) for w in workloads], indent=1)


def loads(text: str) -> list:
    data = json.loads(text)
    if isinstance(data, dict):
        data = [data]
    names = {f.name for f in dataclasses.fields(Workload)}
    out = []
    for d in data:
        unknown = set(d) - names
        if unknown:
            raise ValueError(f"unknown workload field(s) {sorted(unknown)}")
        out.append(Workload(**d))
    return out


def load(path: str) -> list:
    with open(path) as f:
        return loads(f.read())
