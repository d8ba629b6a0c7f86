"""Full-step parity on the benchmark's own workload family (FP32 mixed path,
dynamic steps with slip) and on two targeted contact cases, against the FP64
oracle.  The oracle runs (tests/oracle_cases.py) start at once in spawned
worker processes, one per case, while the GPU runs the same cases; each test
then waits for its case.

Checked at the state the GPU reached after the same poses: positions within
1e-3 of the indentation depth of the oracle's, total contact force within
0.5 %, sigma (relative Frobenius) within 1e-4 and the pressure map (relative
L2) within 1e-3 of the oracle's evaluation at the GPU positions, and the GPU
state penetration-free by the oracle's exact test."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle_cases as oc
from gpu_util import rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oracle_runs():
    # spawned (not forked) workers: this process already holds a CUDA context
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(len(oc.CASES))
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    runs = {name: pool.apply_async(oc.run_case, (name,)) for name in oc.CASES}
    yield runs
    pool.terminate()
    pool.join()


def _gpu_run(name, precision):
    from paper_2606_20426_gb300 import Env
    env = oc.build_case(name)
    g = Env(env, precision=precision)
    for k in range(oc.STEPS[name]):
        g.step(env["poses"][k])
    return env, g


def _check(env, g, ref):
    x = g.positions()
    depth = env["depth"]
    dx = np.abs(x - ref.x).max()
    assert dx <= 1e-3 * depth, f"positions differ by {dx:.3e} m (depth {depth:.3e})"
    f, fr = g.contact_force(), ref.contact_force()
    assert np.linalg.norm(fr) > 0
    assert np.linalg.norm(f - fr) <= 5e-3 * np.linalg.norm(fr), (f, fr)
    assert rel_fro(g.stress().cpu().numpy().T, ref.stress(x)) <= 1e-4
    m, mask = g.pressure_map()
    mref, mask_ref = ref.pressure_map(x=x)
    assert np.array_equal(mask.cpu().numpy(), mask_ref)
    assert rel_fro(m.cpu().numpy(), mref) <= 1e-3
    assert ref.separated(x, ref.indenter(ref.pose))
    return x


@pytest.mark.parametrize("name", ["pad-sphere", "pad-cylinder", "pad-box"])
def test_graded_pad_three_dynamic_steps_each_indenter(oracle_runs, name):
    env, g = _gpu_run(name, "fp32")
    ref = oracle_runs[name].get(timeout=560)
    _check(env, g, ref)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graded_pad_with_friction(oracle_runs, precision):
    """Lagged IPC friction (ratio 0.5, threshold 0.01 m/s) under a sliding
    sphere: the total contact force, tangential part included, matches the
    oracle within 0.5 %, and the friction really acts (its tangential force
    is a sizeable fraction of mu times the normal force)."""
    env, g = _gpu_run("pad-friction", precision)
    ref = oracle_runs["pad-friction"].get(timeout=560)
    _check(env, g, ref)
    f = g.contact_force()
    assert np.hypot(f[0], f[1]) > 0.2 * 0.5 * abs(f[2])
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dual_layer_block(oracle_runs, precision):
    """Heterogeneous (per-tet) material: a soft 1.5 mm top layer (0.3 MPa) on
    a stiff base (1.2 MPa)."""
    env, g = _gpu_run("dual-layer", precision)
    ref = oracle_runs["dual-layer"].get(timeout=560)
    _check(env, g, ref)
    g.close()


def test_bench_env_first_step(oracle_runs):
    """The 59,220-tet env the benchmark steps (seed 0, a cylinder), its first
    load pose, FP32 mixed."""
    env, g = _gpu_run("bench-59k", "fp32")
    assert g.info["nt"] == 59220
    ref = oracle_runs["bench-59k"].get(timeout=560)
    _check(env, g, ref)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pairs_below_one_hundredth_of_dhat(oracle_runs, precision):
    """Soft barrier: the converged contact pairs sit below 1e-2 dhat, where
    the mixed path evaluates the pair distance in FP64."""
    env, g = _gpu_run("close-pairs", precision)
    ref = oracle_runs["close-pairs"].get(timeout=560)
    x = _check(env, g, ref)
    assert oc.min_pair_distance(ref, x) < 1e-2 * env["opts"]["dhat"]
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_parallel_edges_mollifier_active(oracle_runs, precision):
    """A cylinder lying along the pad's grid lines: gel and indenter edges are
    exactly parallel, and the edge-edge mollifier is active."""
    env, g = _gpu_run("parallel-edges", precision)
    ref = oracle_runs["parallel-edges"].get(timeout=560)
    x = _check(env, g, ref)
    assert oc.parallel_ee_pairs(ref, x) >= 1
    g.close()
