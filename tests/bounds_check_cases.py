"""Cases run against the bounds-checked debug build of the library
(libclbm_bc.so, loaded when CLBM_LIBRARY=bounds_check): every index a step or
state kernel derives from the streaming maps or a staged tile is checked
against its buffer, and clbm_check raises CLBM_ERR_BOUNDS after any
violation. Run as a script by test_gpu_bounds_check.py; prints one JSON line
per case and exits non-zero if any case fails."""
import json
import os
import sys
import traceback

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from gpu_common import F32_REL_TOL, W, dev, gpu_f, make_pair, rel_err, t  # noqa: E402
from paper_1801_04586_gb300 import Lattice, _capi, synthetic  # noqa: E402

RATES = dict(s2b=1.2, s3=1.1, s4=0.9)

DEGENERATE = [((1, 1, 1), 0), ((1, 1, 1), 7), ((1, 1, 40), 4), ((5, 1, 1), 0), ((2, 3, 2), 7), ((64, 1, 3), 2),
              ((65535, 1, 1), 1), ((1, 65535, 1), 0), ((1, 1, 65535), 4), ((150, 20, 12), 7)]


def degenerate(shape_xyz, walls):
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    g, o = make_pair(nx, ny, nz, 0.1, walls=walls, s2b=0.9, s3=1.2)
    h0 = synthetic.random_deviations(shape, 1e-3, seed=41)
    F = synthetic.gaussian_force(shape, 1e-5, seed=42)
    g.set_force_field(t(F))
    g.set_populations(t(h0), deviation=True)
    g.step(30)
    g.check()
    fo = oracle.step(o, h0.astype(np.float64) + W, F, 30)
    err = rel_err(gpu_f(g), fo)
    g.close()
    assert err < F32_REL_TOL, err
    return {"rel": err}


def staged(shape_xyz, walls, storage, lattice=19):
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    outs = []
    for variant in (0, 1):
        kw = dict(s3b=1.3, s4b=0.8, s5=1.15, s6=0.95) if lattice == 27 else {}
        g = Lattice(nx, ny, nz, 0.02, walls=walls, storage=storage, variant=variant, lattice=lattice, device=dev(),
                    **RATES, **kw)
        assert g.info()["staged"] == (1 if variant == 0 else 0)
        g.set_force_field(t(synthetic.gaussian_force(shape, 1e-4, seed=503)))
        g.init_equilibrium(None, t(synthetic.divfree_velocity(shape, seed=502, umax=0.04)))
        g.step(5)
        g.check()
        outs.append(g.populations(deviation=True).cpu())
        g.close()
    assert torch.equal(outs[0], outs[1])
    return {}


def in_place(shape_xyz, walls, storage, lattice=19, variant=1):
    """The in-place pattern (variant 0: staged in node pairs for 16-bit D3Q19)
    against the one-node A/B step."""
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    outs = []
    for pattern in ("aa", "ab"):
        g = Lattice(nx, ny, nz, 0.03, walls=walls, storage=storage, pattern=pattern, lattice=lattice,
                    variant=variant if pattern == "aa" else 1, device=dev(), **RATES)
        if pattern == "aa":
            assert g.info()["staged"] == (1 if variant == 0 else 0)
        g.set_force_field(t(synthetic.gaussian_force(shape, 1e-4, seed=61)))
        g.init_equilibrium(None, t(synthetic.divfree_velocity(shape, seed=62, umax=0.03)))
        g.step(7)
        g.check()
        outs.append(g.populations(deviation=True).cpu())
        g.close()
    assert torch.equal(outs[0], outs[1])
    return {}


def slabs_case(storage="f32"):
    nx, ny, nz = 24, 10, 9
    shape = (nz, ny, nx)
    u0 = synthetic.divfree_velocity(shape, seed=5, umax=0.03)
    ranges = [(0, 1), (1, 5), (5, 9)]
    lats = []
    for z0, z1 in ranges:
        lat = Lattice(nx, ny, z1 - z0, 0.04, walls=2, storage=storage, device=dev(), slab=3, z0=z0, **RATES)
        lat.init_equilibrium(None, t(np.ascontiguousarray(u0[:, z0:z1])))
        lats.append(lat)
    for _ in range(6):
        for lat in lats:
            lat.slab_step()
        faces = [lat.faces() for lat in lats]
        for r in range(3):
            half = faces[r][0].numel() // 2
            faces[(r + 1) % 3][1][:half].copy_(faces[r][0][half:])
            faces[(r - 1) % 3][1][half:].copy_(faces[r][0][:half])
    for lat in lats:
        lat.populations()
        lat.macros()
        lat.reduce_moments()
        lat.check()
        lat.close()
    return {}


CASES = [("degenerate", degenerate, c) for c in DEGENERATE] + [
    ("staged", staged, ((64, 20, 9), 0, "f16")),
    ("staged", staged, ((40, 33, 7), 6, "bf16sr")),
    ("staged", staged, ((8, 70, 5), 7, "f16sr")),
    ("staged", staged, ((1024, 3, 4), 2, "f16")),
    ("staged", staged, ((256, 1, 3), 0, "bf16")),
    ("staged", staged, ((24, 50, 1), 4, "f16")),
    ("staged", staged, ((48, 16, 16), 1, "f16")),
    ("staged", staged, ((32, 20, 6), 6, "f16", 27)),
    ("in_place", in_place, ((13, 7, 5), 7, "f32")),
    ("in_place", in_place, ((16, 9, 4), 0, "f16sr")),
    ("in_place", in_place, ((9, 6, 5), 3, "f32", 27)),
    ("in_place", in_place, ((48, 30, 10), 7, "f16sr", 19, 0)),
    ("in_place", in_place, ((8, 130, 3), 0, "bf16", 19, 0)),
    ("slabs", slabs_case, ()),
    ("slabs", slabs_case, ("f16sr",)),
]


def main():
    assert os.environ.get("CLBM_LIBRARY") == "bounds_check"
    assert _capi.lib()._name.endswith("libclbm_bc.so")
    failed = 0
    for name, fn, args in CASES:
        try:
            out = fn(*args)
            print(json.dumps({"case": name, "args": str(args), "ok": True, **out}), flush=True)
        except Exception:
            failed += 1
            print(json.dumps({"case": name, "args": str(args), "ok": False, "error": traceback.format_exc()[-800:]}),
                  flush=True)
    return 1 if failed else 0


if __name__ == "__main__":
    sys.exit(main())
