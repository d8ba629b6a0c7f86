"""GPU parity of the full step (rows a1-a9, a14) against the FP64 oracle.

After converged steps: positions within 1e-3 of the indentation depth,
total contact force within 0.5 %, sigma (relative Frobenius) within 1e-4 and
the pressure map within 1e-3 evaluated on the GPU's own positions; plus the
error paths (initial penetration, non-finite pose, inverted tet)."""
import copy

import numpy as np
import pytest

from gpu_util import rel_fro
from oracle.sim import Scene
from synth import workloads

pytestmark = pytest.mark.gpu


def _run(env, precision, nsteps):
    from paper_2606_20426_gb300 import Env
    g = Env(env, precision=precision)
    ref = Scene(env)
    for k in range(nsteps):
        g.step(env["poses"][k])
        ref.step(env["poses"][k])
    return g, ref


def _check(env, g, ref):
    x = g.positions()
    depth = env["depth"]
    assert np.abs(x - ref.x).max() <= 1e-3 * depth
    f, fr = g.contact_force(), ref.contact_force()
    assert np.linalg.norm(f - fr) <= 5e-3 * np.linalg.norm(fr)
    assert rel_fro(g.stress().cpu().numpy().T, ref.stress(x)) <= 1e-4
    m, _ = g.pressure_map()
    mref, _ = ref.pressure_map(x=x)
    assert rel_fro(m.cpu().numpy(), mref) <= 1e-3
    # the GPU state is penetration-free and in equilibrium per the oracle
    assert ref.separated(x, ref.indenter(ref.pose))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", [0, 5])
def test_small_quasistatic(precision, seed):
    env = workloads.small_env(seed)
    g, ref = _run(env, precision, len(env["poses"]))
    _check(env, g, ref)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small_dynamic(precision):
    env = workloads.small_env(4, dt=1.0 / 60.0)
    g, ref = _run(env, precision, 2)
    _check(env, g, ref)
    g.close()


def test_pad1800_two_steps_fp64():
    env = workloads.pad_env(1, steps=2)
    g, ref = _run(env, "fp64", 2)
    _check(env, g, ref)
    g.close()


def test_initial_penetration_rejected():
    from paper_2606_20426_gb300 import Env, TcError
    env = copy.deepcopy(workloads.small_env(0))
    env["start_pose"]["t"] = env["start_pose"]["t"] - np.array([0, 0, 0.5e-3])
    with pytest.raises(TcError) as ei:
        Env(env)
    assert ei.value.code == 3


def test_nonfinite_pose_rejected():
    from paper_2606_20426_gb300 import Env, TcError
    env = workloads.small_env(0)
    g = Env(env)
    bad = copy.deepcopy(env["poses"][0])
    bad["t"][2] = np.nan
    with pytest.raises(TcError) as ei:
        g.step(bad)
    assert ei.value.code == 7
    g.step(env["poses"][0])  # the env is still usable
    g.close()


def test_inverted_tet_rejected():
    from paper_2606_20426_gb300 import Env, TcError
    env = copy.deepcopy(workloads.small_env(0))
    env["tets"][7, [1, 2]] = env["tets"][7, [2, 1]]
    with pytest.raises(TcError) as ei:
        Env(env)
    assert ei.value.code == 2
