"""GPU parity of the lagged IPC friction (friction ratio 0.5 and velocity
threshold 0.01 m/s of Sec. III-B) against the FP64 oracle, on a small pad
dragged by a sphere; an env with friction gives the same result alone and
in a batch with frictionless envs; friction off leaves the frictionless path
unchanged."""
import copy

import numpy as np
import pytest

from gpu_util import rel_fro
from oracle.sim import Scene
from synth import workloads

pytestmark = pytest.mark.gpu


def _dragged(mu, seed=4, steps=3):
    env = copy.deepcopy(workloads.small_env(seed, dt=1.0 / 60.0, steps=steps))
    for k, p in enumerate(env["poses"]):
        p["t"] = p["t"] + np.array([0.2e-3 * (k + 1), 0.05e-3 * (k + 1), 0.0])
    env["opts"]["friction_mu"] = mu
    env["opts"]["friction_eps_v"] = 0.01
    return env


@pytest.fixture(scope="module")
def oracle_dragged():
    env = _dragged(0.5)
    ref = Scene(env)
    for p in env["poses"]:
        ref.step(p)
    return env, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_friction_step_matches_oracle(oracle_dragged, precision):
    from paper_2606_20426_gb300 import Env
    env, ref = oracle_dragged
    g = Env(env, precision=precision)
    for p in env["poses"]:
        g.step(p)
    x = g.positions()
    assert np.abs(x - ref.x).max() <= 1e-3 * env["depth"]
    f, fr = g.contact_force(), ref.contact_force()
    assert np.hypot(fr[0], fr[1]) > 0.3 * 0.5 * abs(fr[2])      # the drag is carried by friction
    assert np.linalg.norm(f - fr) <= 5e-3 * np.linalg.norm(fr), (f, fr)
    assert rel_fro(g.stress().cpu().numpy().T, ref.stress(x)) <= 1e-4
    m, _ = g.pressure_map()
    assert rel_fro(m.cpu().numpy(), ref.pressure_map(x=x)[0]) <= 1e-3
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_friction_env_alone_equals_batched(precision):
    from paper_2606_20426_gb300 import Env, step_batch
    cfgs = [_dragged(0.5, seed=4), _dragged(0.0, seed=5), _dragged(0.3, seed=6)]
    alone = [Env(c, precision=precision) for c in cfgs]
    batch = [Env(c, precision=precision) for c in cfgs]
    for k in range(3):
        for g, c in zip(alone, cfgs):
            g.step(c["poses"][k])
        assert step_batch(batch, [c["poses"][k] for c in cfgs]) == [0, 0, 0]
    for a, b in zip(alone, batch):
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.contact_force(), b.contact_force())
    for g in alone + batch:
        g.close()


def test_zero_friction_is_the_frictionless_path():
    """friction_mu = 0 (and friction in a quasi-static scene) computes exactly
    what the scene without the friction options computes."""
    from paper_2606_20426_gb300 import Env
    a_cfg = _dragged(0.0)
    b_cfg = copy.deepcopy(a_cfg)
    del b_cfg["opts"]["friction_mu"], b_cfg["opts"]["friction_eps_v"]
    q_cfg = copy.deepcopy(workloads.small_env(0, steps=2))
    q_cfg["opts"]["friction_mu"] = 0.5
    q_ref = workloads.small_env(0, steps=2)
    for c1, c2 in ((a_cfg, b_cfg), (q_cfg, q_ref)):
        g1, g2 = Env(c1, precision="fp32"), Env(c2, precision="fp32")
        for p in c1["poses"]:
            g1.step(p)
            g2.step(p)
        assert np.array_equal(g1.positions(), g2.positions())
        g1.close()
        g2.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vertex_forces_and_force_pressure_map(oracle_dragged, precision):
    """Algorithm 2's per-vertex decomposition (f, f_n, f_tau, p = |f|/A) and
    its pixel map, friction included, against the oracle's at the GPU state."""
    from paper_2606_20426_gb300 import Env
    env, ref = oracle_dragged
    g = Env(env, precision=precision)
    for p_ in env["poses"]:
        g.step(p_)
    x = g.positions()
    f, fn, ft, p = (t.cpu().numpy().astype(np.float64) for t in g.vertex_forces())
    rf, rfn, rft, rp, _, _ = ref.vertex_contact_forces(x)
    scale = np.abs(rf).max()
    # the oracle's friction terms at the GPU state use the oracle's own lagged
    # normal forces (from its own converged substeps), so per-vertex forces
    # agree to the accuracy of the states, not to rounding
    tol = 1e-3 if precision == "fp32" else 1e-4
    assert np.abs(f.T - rf).max() <= tol * scale
    assert np.abs(fn.T - rfn).max() <= tol * scale and np.abs(ft.T - rft).max() <= tol * scale
    assert np.abs(p - rp).max() <= tol * np.abs(rp).max()
    assert np.abs(f.sum(axis=1) - g.contact_force()).max() <= 1e-4 * scale
    m, mask = g.force_pressure_map()
    mref, mask_ref = ref.pressure_map(p_vertex=rp)
    assert np.array_equal(mask.cpu().numpy(), mask_ref)
    assert rel_fro(m.cpu().numpy(), mref) <= 1e-3
    g.close()
