"""The bounds-checked build (libbt_checked.so, -DBT_CHECKED) against the
normal one.

The checked build tests every shared-memory, gather and output index the
residual pass forms before the access and reports a failed test as
BT_ERR_INVALID instead of faulting -- the stand-in for a memory checker.
The same solves (single graphs of both resolutions and a batch) run through
both libraries in separate processes; no test may fail and the results must
be identical (the tests add branches, not arithmetic)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[2])
import numpy as np
import synthgen as S
from paper_2108_00516_gb300 import bt
bt.load(sys.argv[1])
out = {}
for k in range(3):
    g = S.tiny_graph(k)
    pg = bt.graph_from_synth(g)
    P, r = pg.solve(5)
    out["tiny%d" % k] = [P.ravel().tolist(), r["cost_final"], r["dense_inliers"], pg.eval_cost()["total"]]
g = S.paper_graph(0, n_frames=4)
pg = bt.graph_from_synth(g)
P, r = pg.solve(3)
out["paper"] = [P.ravel().tolist(), r["cost_final"], r["dense_inliers"]]
gs = [S.tiny_graph(k) for k in range(3, 6)] + [S.random_graph(4321, 5, S.QVGA_CAMERA, 300, 0.2, coverage_target=0.12)]
pgs = [bt.graph_from_synth(x) for x in gs]
b = bt.Batch()
for x in pgs:
    b.add(x)
b.set_shape(3)
reps = b.solve(4)
out["batch"] = [[x.get_poses().ravel().tolist() for x in pgs], [r["cost_final"] for r in reps]]
print(json.dumps(out))
"""


def _run(lib):
    r = subprocess.run([sys.executable, "-c", SCRIPT, str(lib), ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_matches_normal_build():
    from paper_2108_00516_gb300 import build as lbuild
    normal = lbuild.build()
    checked = lbuild.build(checked=True)
    a = _run(normal)
    b = _run(checked)
    assert a == b
