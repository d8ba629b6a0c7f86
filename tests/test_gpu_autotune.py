"""PCG launch-shape selection: tc_autotune_pcg times every co-schedulable
shape on the envs' current Newton systems (latency and throughput modes)
without moving the envs, selects one, and stepping afterwards still matches
the oracle; tc_pcg_shape rejects shapes outside 1..16 CTAs x {512, 1024}
threads, and clusters of 12 and 3 CTAs (non-power-of-two splits of the rows)
give the oracle's state too."""
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
        pcg_shape("fp32", 0, 1024)
    with pytest.raises(TcError):
        pcg_shape("fp32", 17, 1024)
    with pytest.raises(TcError):
        pcg_shape("fp32", 16, 256)
    _restore_default()


@pytest.mark.parametrize("cs", [12, 3])
def test_odd_cluster_sizes_match_oracle(cs):
    """Cluster sizes that are not powers of two split the rows unevenly; the
    solve still reaches the oracle's state (FP32 mixed path, two steps)."""
    from paper_2606_20426_gb300 import Env, TcError, pcg_shape
    s = workloads.small_env(3)
    try:
        try:
            pcg_shape("fp32", cs, 1024)
        except TcError:
            pytest.skip(f"a {cs}-CTA cluster of 1024 threads cannot be co-scheduled here")
        g = Env(s, precision="fp32")
        ref = Scene(s)
        for k in range(2):
            g.step(s["poses"][k])
            ref.step(s["poses"][k])
        assert np.abs(g.positions() - ref.x).max() <= 1e-3 * s["depth"]
        g.close()
    finally:
        _restore_default()
