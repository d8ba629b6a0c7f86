"""GPU parity of the full stable Neo-Hookean law (log term,
TC_MODEL_SNH_LOG) against the FP64 oracle: the incremental potential and its
gradient at an in-contact state, sigma at given positions (including large
strains), and full steps (quasi-static and dynamic, FP64 and FP32 mixed)
under the same tolerances as the rest-stable law: positions within 1e-3 of
the depth, contact force within 0.5 %, sigma within 1e-4 and the pressure
map within 1e-3 at the GPU's positions."""
import copy

import numpy as np
import pytest

from gpu_util import rel_fro
from oracle.sim import Scene
from synth import workloads

pytestmark = pytest.mark.gpu


def _log(env):
    env = copy.deepcopy(env)
    env["material"] = dict(env["material"], model="snh_log")
    return env


@pytest.mark.parametrize("precision,etol,gtol", [("fp64", 1e-10, 1e-9), ("fp32", 1e-5, 2e-3)])
def test_energy_gradient_in_contact(precision, etol, gtol):
    from paper_2606_20426_gb300 import Env
    env = _log(workloads.small_env(0))
    ref = Scene(env)
    ref.step(env["poses"][0])
    rng = np.random.default_rng(3)
    x = ref.x + 1e-3 * env["opts"]["dhat"] * rng.standard_normal(ref.x.shape) * ref.free[:, None]
    Y = ref.indenter(env["poses"][0])
    Eref = ref.energy(x, Y, ref.candidates(x, Y))
    _, gref, _ = ref.gradient_hessian(x, Y)
    gref = gref.reshape(-1, 3)
    gref[~ref.free] = 0.0
    g = Env(env, precision=precision)
    g.step(env["poses"][0])
    g.set_positions(x)
    E, grad = g.energy_gradient()
    g.close()
    assert abs(E - Eref) <= etol * abs(Eref)
    assert rel_fro(grad, gref) <= gtol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("amp", [2e-5, 1.5e-4])
def test_stress_at_given_positions(precision, amp):
    """sigma of every tet at positions displaced randomly (strains up to
    ~7 % and ~55 %, where the log term is far from its linearisation)."""
    from paper_2606_20426_gb300 import Env
    env = _log(workloads.small_env(1))
    ref = Scene(env)
    rng = np.random.default_rng(int(amp * 1e6))
    x = ref.X + amp * rng.standard_normal(ref.X.shape) * ref.free[:, None]
    g = Env(env, precision=precision)
    g.set_positions(x)
    s = g.stress().cpu().numpy().T.astype(np.float64)
    g.close()
    assert rel_fro(s, ref.stress(x)) <= 1e-4


def _steps(env, precision, n):
    from paper_2606_20426_gb300 import Env
    g = Env(env, precision=precision)
    ref = Scene(env)
    for k in range(n):
        g.step(env["poses"][k])
        ref.step(env["poses"][k])
    x = g.positions()
    assert np.abs(x - ref.x).max() <= 1e-3 * env["depth"]
    f, fr = g.contact_force(), ref.contact_force()
    assert np.linalg.norm(f - fr) <= 5e-3 * np.linalg.norm(fr)
    assert rel_fro(g.stress().cpu().numpy().T, ref.stress(x)) <= 1e-4
    m, _ = g.pressure_map()
    mref, _ = ref.pressure_map(x=x)
    assert rel_fro(m.cpu().numpy(), mref) <= 1e-3
    assert ref.separated(x, ref.indenter(ref.pose))
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small_quasistatic(precision):
    env = _log(workloads.small_env(0))
    _steps(env, precision, len(env["poses"]))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_small_dynamic(precision):
    env = _log(workloads.small_env(4, dt=1.0 / 60.0))
    _steps(env, precision, 2)


def test_dual_layer_with_log_law():
    """Per-tet (E, nu) under the log law: a two-layer table on a small pad."""
    env = _log(workloads.small_env(5))
    Z = np.asarray(env["X"])[np.asarray(env["tets"])].mean(axis=1)[:, 2]
    top = Z > np.median(Z)
    env["material"]["per_tet"] = np.stack([np.where(top, 3.0e5, 1.2e6), np.full(len(Z), 0.45)], axis=1)
    _steps(env, "fp64", len(env["poses"]))


def test_unknown_model_is_rejected():
    from paper_2606_20426_gb300 import Env
    env = copy.deepcopy(workloads.small_env(0))
    env["material"] = dict(env["material"], model="mooney")
    with pytest.raises(ValueError):
        Env(env)
