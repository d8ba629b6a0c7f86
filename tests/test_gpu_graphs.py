"""CUDA-graph replay of the phase launch sequences leaves results unchanged:
the same envs stepped in a process with graphs and in one without
(TACAUCHY_GRAPHS=0) end bit-identical in positions, stress and contact
force, and take the same Newton and CG iterations."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from synth import workloads
from paper_2606_20426_gb300 import Env, step_batch
out = {}
for precision in ("fp32", "fp64"):
    scenes = [workloads.small_env(0, steps=6), workloads.small_env(4, steps=6, dt=1.0 / 60.0)]
    envs = [Env(s, precision=precision) for s in scenes]
    for k in range(3):
        for s, e in zip(scenes, envs):      # one env per launch
            e.step(s["poses"][k])
    for k in range(3, len(scenes[0]["poses"])):
        assert step_batch(envs, [s["poses"][k] for s in scenes]) == [0, 0]   # both in one batch
    for i, e in enumerate(envs):
        inf = e.get_info()
        out[f"{precision}{i}"] = dict(x=e.positions().tolist(), s=e.stress().cpu().numpy().tolist(),
                                      f=list(e.contact_force()), n=inf["newton_iters"], c=inf["pcg_iters"])
        e.close()
json.dump(out, open(sys.argv[2], "w"))
"""


def _run(tmp_path, graphs):
    path = str(tmp_path / f"out_{graphs}.json")
    env = dict(os.environ, TACAUCHY_GRAPHS=graphs, TACAUCHY_TRACE="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, path], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.load(open(path)), r.stderr.count("captured")


def test_graph_replay_is_bit_identical(tmp_path):
    a, na = _run(tmp_path, "1")
    b, nb = _run(tmp_path, "0")
    assert na > 0 and nb == 0  # graphs were captured (and replayed) in the first run only
    assert a.keys() == b.keys()
    for k in a:
        assert a[k]["n"] == b[k]["n"] and a[k]["c"] == b[k]["c"], k
        for f in ("x", "s", "f"):
            assert np.array_equal(np.asarray(a[k][f]), np.asarray(b[k][f])), (k, f)
