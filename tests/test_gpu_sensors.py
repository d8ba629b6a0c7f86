"""Dome (DIGIT-like) and block (9DTact-like) sensors: parity of a converged
step against the FP64 oracle on small meshes, and an uneven batch of a pad,
a dome and a block whose envs end bit-identical to the same envs stepped
alone (one launch per Newton phase over meshes of different sizes)."""
import numpy as np
import pytest

from gpu_util import rel_fro
from oracle.sim import Scene
from synth import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sensor", ["dome", "block"])
def test_sensor_step_matches_oracle(sensor):
    from paper_2606_20426_gb300 import Env
    env = workloads.sensor_env(3, sensor, 1000, steps=3, dt=0.0, precision="fp64", pixel=0.5e-3)
    g = Env(env, precision="fp64")
    ref = Scene(env)
    for k in range(1):
        g.step(env["poses"][k])
        ref.step(env["poses"][k])
    x = g.positions()
    assert np.abs(x - ref.x).max() <= 1e-3 * env["depth"]
    f, fr = g.contact_force(), ref.contact_force()
    assert np.linalg.norm(f - fr) <= 5e-3 * max(np.linalg.norm(fr), 1e-12)
    assert rel_fro(g.stress().cpu().numpy().T, ref.stress(x)) <= 1e-4
    m, _ = g.pressure_map()
    mref, _ = ref.pressure_map(x=x)
    assert rel_fro(m.cpu().numpy(), mref) <= 1e-3
    assert ref.separated(x, ref.indenter(ref.pose))
    g.close()


def test_uneven_sensor_batch_equals_alone():
    from paper_2606_20426_gb300 import Env, step_batch
    scenes = [workloads.sensor_env(11, "pad", 5000, steps=2), workloads.sensor_env(12, "dome", 8000, steps=2),
              workloads.sensor_env(13, "block", 10000, steps=2)]
    batch = [Env(s, precision="fp32") for s in scenes]
    for k in range(2):
        assert step_batch(batch, [s["poses"][k] for s in scenes]) == [0, 0, 0]
    for s, g in zip(scenes, batch):
        a = Env(s, precision="fp32")
        for k in range(2):
            a.step(s["poses"][k])
        assert np.array_equal(g.positions(), a.positions())
        assert np.array_equal(g.stress().cpu().numpy(), a.stress().cpu().numpy())
        assert np.array_equal(g.pressure_map()[0].cpu().numpy(), a.pressure_map()[0].cpu().numpy())
        a.close()
        g.close()
