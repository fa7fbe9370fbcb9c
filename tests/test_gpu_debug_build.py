"""The bounds-checked build (TLSPH_DEBUG): every neighbour index the kernels use is checked against the
particle range (stencil slots may point into the zero halo, active neighbours may not).  The same cases
run through it in a child process (the binding loads one library per process, chosen by TLSPH_LIBRARY)
must step without a flag and match the release build bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2602_15149_b300 import build, tlsph, workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
from paper_2602_15149_b300 import tlsph, workloads as W
cases = {"block_stencil": lambda: W.block_3d(nx=16, ny=12, nz=10),
         "notched_phase_field": lambda: W.notched_plate(nx=60, ny=24, model="svk"),
         "batched_tables": lambda: W.batched(nspec=12, n_min=40, n_max=400, seed=3),
         "irregular_csr": lambda: W.block_3d(nx=9, ny=8, nz=7, jitter=0.3, seed=5),
         "contact": lambda: W.flyer_plate(n=10, dx=1e-3, gap=0.0, v=2.0, model="nh", precision="fp64"),
         "lattice_zstream": lambda: W.block_3d(nx=24, ny=20, nz=16),
         "lattice_patch": lambda: W.block_3d(nx=40, ny=9, nz=7)}
options = {"lattice_zstream": {tlsph.OPT_LATTICE_ZSTREAM: 5},
           "lattice_patch": {tlsph.OPT_LATTICE_PATCH: 32, tlsph.OPT_LATTICE_ROWS_FORCE: 4}}
out = {}
for name, make in cases.items():
    g = tlsph.from_case(make())
    for k, v in options.get(name, {}).items():
        g.set_option(k, v)
    st = g.step(100, check=False)
    out[name] = {"status": int(st), "u": g.read_state("U").tolist(), "stencil": g.get_info()["stencil"]}
print(json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ, TLSPH_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_finds_no_bad_index_and_matches_release():
    dbg = build.build_library(debug=True)
    rel = build.build_library()
    a, b = _run(dbg), _run(rel)
    assert a["irregular_csr"]["stencil"] == 0 and a["block_stencil"]["stencil"] > 0
    for name in a:
        assert a[name]["status"] == tlsph.OK, (name, a[name]["status"])
        assert np.array_equal(np.array(a[name]["u"]), np.array(b[name]["u"])), name
