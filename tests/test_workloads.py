"""The workload descriptions (paper_1801_04586_gb300/workloads) load into
their dataclass, and the benchmark runs what they state."""
import importlib.util
import os

import pytest

from paper_1801_04586_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_workload_loads():
    assert workloads.names() == ["adjoint_force_64", "batch_64_domains", "duct_mixed_precision",
                                 "kolmogorov_256", "poiseuille_channel"]
    for name in workloads.names():
        w = workloads.load(name)
        assert w.name == name and w.what and w.steps > 0
        assert w.storage in ("f32", "f16", "bf16", "f16sr", "bf16sr") and w.pattern in ("ab", "aa")
        if w.domains is None:
            assert w.nodes > 0 and 0 < w.nu and w.walls in range(8)
            kw = w.lattice_kwargs()
            assert (kw["nx"], kw["ny"], kw["nz"]) == (w.nx, w.ny, w.nz)
        else:
            with pytest.raises(ValueError):
                w.lattice_kwargs()
    with pytest.raises(KeyError):
        workloads.load("no_such_workload")


def test_benchmark_runs_the_stated_workloads():
    b = _bench()
    k = workloads.load("kolmogorov_256")
    assert (k.nx, k.ny, k.nz) == (b.N_SIDE,) * 3 and k.nu == b.NU and k.force["F0"] == b.F0
    assert "0.02" in k.init["u"] and b.UMAX == 0.02
    d = workloads.load("duct_mixed_precision")
    assert (d.nx, d.ny, d.nz, d.walls, d.nu, d.force["fx"]) == (512, 128, 128, 6, 0.05, 2e-6)
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert "Lattice(512, 128, 128, 0.05, walls=6" in src and "set_force_uniform(2e-6)" in src
    bt = workloads.load("batch_64_domains")
    assert "batch_domains(64, seed=6)" in src and (bt.domains["count"], bt.domains["seed"]) == (64, 6)
