"""Batched steps (tc_step_batch): every env in a batch ends bit-identical to
the same env stepped alone with tc_step, for envs of different sizes, both
precisions and a quasistatic/dynamic mix; a bad pose fails only its own env;
the argument checks of the batch call."""
import copy

import numpy as np
import pytest

from synth import workloads

pytestmark = pytest.mark.gpu


def _alone(env, precision, nsteps):
    from paper_2606_20426_gb300 import Env
    g = Env(env, precision=precision)
    for k in range(nsteps):
        g.step(env["poses"][k])
    return g


def _same(a, b):
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.stress().cpu().numpy(), b.stress().cpu().numpy())
    assert np.array_equal(a.contact_force(), b.contact_force())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_alone(precision):
    from paper_2606_20426_gb300 import Env, step_batch
    scenes = [workloads.small_env(0), workloads.small_env(5), workloads.pad_env(1, steps=2),
              workloads.small_env(4, dt=1.0 / 60.0)]
    nsteps = 2
    batch = [Env(s, precision=precision) for s in scenes]
    for k in range(nsteps):
        codes = step_batch(batch, [s["poses"][k] for s in scenes])
        assert codes == [0] * len(scenes)
    for s, g in zip(scenes, batch):
        alone = _alone(s, precision, nsteps)
        _same(g, alone)
        assert g.get_info()["newton_iters"] == alone.get_info()["newton_iters"]
        alone.close()
        g.close()


def test_batch_of_one_equals_step():
    from paper_2606_20426_gb300 import Env, step_batch
    s = workloads.small_env(0)
    a, b = Env(s), Env(s)
    for k in range(len(s["poses"])):
        a.step(s["poses"][k])
        assert step_batch([b], [s["poses"][k]]) == [0]
    _same(a, b)
    a.close()
    b.close()


def test_bad_pose_fails_only_its_env():
    from paper_2606_20426_gb300 import Env, step_batch
    s0, s1 = workloads.small_env(0), workloads.small_env(5)
    g0, g1 = Env(s0), Env(s1)
    x1 = g1.positions()
    bad = copy.deepcopy(s1["poses"][0])
    bad["t"] = np.array([np.nan, 0.0, 0.0])
    codes = step_batch([g0, g1], [s0["poses"][0], bad])
    assert codes == [0, 7]
    assert np.array_equal(g1.positions(), x1)
    alone = _alone(s0, "fp64", 1)
    _same(g0, alone)
    for g in (g0, g1, alone):
        g.close()


def test_batch_argument_checks():
    from paper_2606_20426_gb300 import Env, TcError, step_batch
    s = workloads.small_env(0)
    a = Env(s, precision="fp64")
    b = Env(s, precision="fp32")
    assert step_batch([], []) == []
    with pytest.raises(TcError) as ei:
        step_batch([a, b], [s["poses"][0]] * 2)
    assert ei.value.code == 1
    with pytest.raises(TcError) as ei:
        step_batch([a, a], [s["poses"][0]] * 2)
    assert ei.value.code == 1
    a.close()
    b.close()
