"""The bounds-checked copy of the library (built with GRMHD_CHECK_BOUNDS): every array
index its kernels form from a grid position or a stride offset is checked against the
padded array, counted when it falls outside and redirected inside.  Run over the
problem set of the parity tests -- every boundary kind, 1-D/2-D/3-D, flat and metric,
MC and PPM, both edge EMFs, CT and GLM, FP64 and mixed precision, the batched
executor, the elliptic cleaning and the diagnostics -- it must count no violation, and
a checked run must still match the oracle.

The checked library is loaded in a child process (the test process has the normal
one loaded)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
from paper_2110_03732_gb300 import build as _b
_b.LIB = _b.LIB_CHECKED
from paper_2110_03732_gb300 import grmhd, problems as P
import numpy as np
import torch
import oracle
from parity_tools import check

assert grmhd.bounds_violations(reset=True) == 0
counts = {}

def run(tag, pr, steps=2, **kw):
    S = grmhd.Solver.from_problem(pr, **kw)
    dt = S.compute_dt()
    for _ in range(steps):
        S.step(dt)
    S.diagnostics()
    counts[tag] = grmhd.bounds_violations(reset=True)
    return S, dt

S, _ = run("ot_periodic", P.orszag_tang(48))
S.clean_divb(2)
S.get_prims()
counts["clean_prims"] = grmhd.bounds_violations(reset=True)
run("box3d_outflow_metric", P.random_box(5, 3, [12, 10, 9], bc="outflow", metric=True))
run("box2d_fixed", P.random_box(7, 2, [20, 14], bc="fixed"))
run("tube1d", P.shock_tube(64), steps=3)
run("glm3d", P.random_box(9, 3, [10, 9, 8], bc="outflow", metric=True, glm=True), divb="glm")
run("ppm2d_fixed", P.random_box(3, 2, [20, 16], bc="fixed"), rec="ppm")
run("ppm3d_periodic", P.random_box(4, 3, [10, 8, 6], bc="periodic"), rec="ppm")
run("ideal2d", P.random_box(2, 2, [18, 16], bc="periodic"), emf="ideal")
run("mixed_ot", P.orszag_tang(32), precision="mixed")
run("star_fp64", P.star(20))
run("star_mixed", P.star(20), precision="mixed")
sol = [grmhd.Solver.from_problem(pr, precision="mixed") for pr in
       (P.shock_tube(80), P.orszag_tang(40), P.random_box(6, 3, [10, 8, 6], bc="outflow", metric=True))]
B = grmhd.Batch(sol)
B.set_dt([s.compute_dt() for s in sol])
for _ in range(2):
    B.step()
counts["batched"] = grmhd.bounds_violations(reset=True)

# a checked run against the oracle (2 steps of the 3-D metric box)
pr = P.random_box(11, 3, [10, 9, 8], bc="outflow", metric=True)
st = oracle.from_problem(pr)
S = grmhd.Solver.from_problem(pr)
dt = S.compute_dt()
for _ in range(2):
    st.step(dt)
    S.step(dt)
torch.cuda.synchronize()
I = st.grid.interior()
for v in range(8):
    check(S.q[v].cpu().numpy()[I], st.q[v][I], f"q[{v}]")
for d in range(3):
    check(S.bf[d].cpu().numpy()[I], st.bf[d][I], f"bf[{d}]")
counts["oracle_box"] = grmhd.bounds_violations(reset=True)
print(json.dumps(counts))
'''


def test_checked_library_counts_no_violation():
    from paper_2110_03732_gb300 import build as _b
    _b.build(checked=True)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    counts = json.loads(r.stdout.strip().splitlines()[-1])
    assert counts and all(v == 0 for v in counts.values()), counts
