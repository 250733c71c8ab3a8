"""The bounds-checked debug build (libclbm_bc.so, -DCLBM_BOUNDS_CHECK) on the
degenerate and ragged lattices of the parity tests, the staged 16-bit tile
shapes, the in-place pattern and the z-slab halo planes: no kernel derives an
index outside its buffer or tile (clbm_check stays CLBM_OK, which in this
build would report CLBM_ERR_BOUNDS), and the results still match the oracle
or the other kernel form bit for bit. Runs the cases of bounds_check_cases.py
in a child process that loads the checked library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_finds_no_out_of_range_index():
    from paper_1801_04586_gb300.builder import build
    build(bounds_check=True)
    env = dict(os.environ, CLBM_LIBRARY="bounds_check")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_check_cases.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    results = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    bad = [x for x in results if not x["ok"]]
    assert not bad, bad
    assert r.returncode == 0, r.stderr[-2000:]
    assert len(results) >= 20
