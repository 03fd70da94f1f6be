"""Autotuned row-kernel shapes and CUDA-graph replay must not change results.

Every shape computes each row's sums in the same order, and a replayed graph runs the
launches it captured, so solves with the tuned shapes, with the default shape
(options autotune=False) and with eager launches (options graphs=False), each in a
child process, give bit-identical eigenvalues and residuals, in both arithmetics."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1511_07042_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json
sys.path.insert(0, sys.argv[1])
from paper_1511_07042_gb300 import bmg, inputs
extra = json.loads(sys.argv[2])
v, t = inputs.icosahedron()
out = {}
for prec, k in (("fp64", 20), ("fp32", 32)):
    p = bmg.Problem(v, t, 4)
    p.hierarchy(4)
    X0 = inputs.gaussian_block(inputs.n_vertices(2), k, 7)
    ev, _, rs, info = p.solve(X0, k, 12, 0.0, 1e-9, bmg.options(precision=prec, **extra), evecs=False)
    out[prec] = [ev.tolist(), rs.tolist(), info.total_cycles]
print(json.dumps({"res": out, "tuned": bmg.autotune_report()}))
"""


def run_child(opts):
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(opts)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tuned_shapes_give_identical_results(gpu_bmg):
    tuned = run_child({})
    plain = run_child({"autotune": False})
    assert tuned["tuned"], "the tuner recorded no shapes"
    assert plain["tuned"] == []
    for prec in ("fp64", "fp32"):
        a, b = tuned["res"][prec], plain["res"][prec]
        assert np.array_equal(np.array(a[0]), np.array(b[0])) and np.array_equal(np.array(a[1]), np.array(b[1]))
        assert a[2] == b[2]
    # every recorded shape covers its block width
    for kind, tb, nch, rows, lanes, chunks, warps in tuned["tuned"]:
        assert lanes * chunks >= nch and warps in (4, 8, 16) and rows > 0


def test_graph_replay_gives_identical_results(gpu_bmg):
    graphs = run_child({})
    eager = run_child({"graphs": False})
    for prec in ("fp64", "fp32"):
        a, b = graphs["res"][prec], eager["res"][prec]
        assert np.array_equal(np.array(a[0]), np.array(b[0])) and np.array_equal(np.array(a[1]), np.array(b[1]))
        assert a[2] == b[2]
