"""The workloads the benchmark and the tests run, as data: one JSON file each
beside this module (the Poiseuille channel of Sec. III.B, the periodic
Kolmogorov throughput box, the mixed-precision square duct of Sec. III.C, the
differentiable forced flow and the 64-domain batch), read into a Workload.

    from paper_1801_04586_gb300 import Lattice, workloads
    w = workloads.load("kolmogorov_256")
    lat = Lattice(**w.lattice_kwargs())

Holds no method arithmetic; the fields are the parameters clbm_params takes
plus the force, the initial state and the step count, stated as data."""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field, fields
from typing import List, Optional

HERE = os.path.dirname(os.path.abspath(__file__))


@dataclass(frozen=True)
class Workload:
    name: str
    what: str
    nx: int = 0
    ny: int = 0
    nz: int = 0
    walls: int = 0              # CLBM_WALL_* bits: 1 x, 2 y, 4 z faces (halfway bounce-back)
    nu: float = 0.0             # kinematic viscosity, s2 = 1/(3 nu + 1/2)
    s2b: float = 1.0
    s3: float = 1.0
    s4: float = 1.0
    force: dict = field(default_factory=dict)   # mode "uniform" / "profile_z" / "field" and its values
    init: dict = field(default_factory=dict)    # initial density and velocity, as described
    storage: str = "f32"        # f32, f16, bf16, f16sr, bf16sr
    pattern: str = "ab"         # ab (two buffers) or aa (in place)
    steps: int = 0
    checkpoint_every: Optional[int] = None      # adjoint unrolls
    domains: Optional[dict] = None              # batches: the draw of the domains

    def lattice_kwargs(self) -> dict:
        """Arguments of Lattice for this workload (single lattices only)."""
        if self.domains is not None:
            raise ValueError(f"{self.name} is a batch: see its domains")
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, nu=self.nu, walls=self.walls, s2b=self.s2b, s3=self.s3,
                    s4=self.s4, storage=self.storage, pattern=self.pattern)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz


def names() -> List[str]:
    return sorted(f[:-5] for f in os.listdir(HERE) if f.endswith(".json"))


def load(name: str) -> Workload:
    path = os.path.join(HERE, name + ".json")
    if not os.path.exists(path):
        raise KeyError(f"no workload {name!r}; known: {', '.join(names())}")
    with open(path) as fh:
        data = json.load(fh)
    known = {f.name for f in fields(Workload)}
    extra = set(data) - known
    if extra:
        raise ValueError(f"{name}: unknown fields {sorted(extra)}")
    return Workload(**data)
