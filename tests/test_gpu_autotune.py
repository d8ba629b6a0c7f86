"""PCG launch-shape selection: tc_autotune_pcg times every co-schedulable
shape on the envs' current Newton systems (latency and throughput modes)
without moving the envs, selects one, and stepping afterwards still matches
the oracle; tc_pcg_shape rejects shapes outside {8, 16} x {512, 1024}."""
import numpy as np
import pytest

from oracle.sim import Scene
from synth import workloads

pytestmark = pytest.mark.gpu


def _restore_default():
    from paper_2606_20426_gb300 import TcError, pcg_shape
    for prec in ("fp32", "fp64"):
        try:
            pcg_shape(prec, 16, 1024)
        except TcError:
            pcg_shape(prec, 8, 1024)


def test_autotune_modes_and_step_after():
    from paper_2606_20426_gb300 import Env, autotune_pcg
    scenes = [workloads.small_env(0), workloads.small_env(5)]
    envs = [Env(s, precision="fp64") for s in scenes]
    for g, s in zip(envs, scenes):
        g.step(s["poses"][0])
    x0 = [g.positions() for g in envs]
    try:
        for mode in ("latency", "throughput"):
            res = autotune_pcg(envs, mode=mode)
            assert len(res) >= 1
            assert all(r["cluster_ctas"] in (8, 16) and r["threads"] in (512, 1024) for r in res)
            assert all(r["env_iters"] > 0 and 0.0 < r["us_per_env_iter"] < 1e6 for r in res)
        for g, x in zip(envs, x0):
            assert np.array_equal(g.positions(), x)  # tuning does not move the envs
        # a step under the selected shape still converges to the oracle's state
        s = scenes[0]
        ref = Scene(s)
        ref.step(s["poses"][0])
        ref.step(s["poses"][1])
        envs[0].step(s["poses"][1])
        assert np.abs(envs[0].positions() - ref.x).max() <= 1e-3 * s["depth"]
    finally:
        for g in envs:
            g.close()
        _restore_default()


def test_shape_argument_checks():
    from paper_2606_20426_gb300 import TcError, pcg_shape
    with pytest.raises(TcError):
        pcg_shape("fp32", 4, 1024)
    with pytest.raises(TcError):
        pcg_shape("fp32", 16, 256)
    _restore_default()
