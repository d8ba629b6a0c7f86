"""Configuration 3 spot check: the 60 uneven envs of the pad / dome / block mix
(5k-80k tets) take one step together (tc_step_batch, one launch per Newton
phase over all of them) and one batched extraction; the two smallest envs of
each family are checked against the FP64 oracle (run in spawned worker
processes while the GPU works): positions within 1e-3 of the indentation
depth, total contact force within 0.5 %, sigma within 1e-4 and the pressure
map within 1e-3 at the GPU state."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from gpu_util import rel_fro

pytestmark = pytest.mark.gpu

PICK = [2, 4, 32, 33, 42, 53]  # the two smallest pads, domes and blocks of mixed_envs(0)


def oracle_first_step(i):
    from oracle.sim import Scene
    from synth import workloads
    env = workloads.mixed_envs(0)[i]
    sc = Scene(env)
    sc.step(env["poses"][0])
    return sc


def test_sixty_env_mix_spot_checks():
    import torch
    from paper_2606_20426_gb300 import Env, extract_batch, step_batch
    from synth import workloads
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    pool = mp.get_context("spawn").Pool(len(PICK))
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    runs = {i: pool.apply_async(oracle_first_step, (i,)) for i in PICK}
    try:
        cfgs = workloads.mixed_envs(0)
        nts = [len(c["tets"]) for c in cfgs]
        assert len(cfgs) == 60 and min(nts) >= 5000 and max(nts) <= 88000
        assert sorted(PICK) == sorted(sorted(range(20), key=nts.__getitem__)[:2] +
                                      sorted(range(20, 40), key=nts.__getitem__)[:2] +
                                      sorted(range(40, 60), key=nts.__getitem__)[:2])
        envs = [Env(c, precision="fp32") for c in cfgs]
        assert step_batch(envs, [c["poses"][0] for c in cfgs]) == [0] * 60
        sig = [torch.empty((6, e.info["nt"]), device="cuda") for e in envs]
        maps = [torch.empty((e.info["H"], e.info["W"]), device="cuda") for e in envs]
        extract_batch(envs, sig, maps, None)
        for i in PICK:
            ref = runs[i].get(timeout=560)
            g, c = envs[i], cfgs[i]
            x = g.positions()
            assert np.abs(x - ref.x).max() <= 1e-3 * c["depth"], (i, np.abs(x - ref.x).max())
            f, fr = g.contact_force(), ref.contact_force()
            assert np.linalg.norm(f - fr) <= 5e-3 * np.linalg.norm(fr), (i, f, fr)
            assert rel_fro(sig[i].cpu().numpy().T, ref.stress(x)) <= 1e-4
            mref, _ = ref.pressure_map(x=x)
            assert rel_fro(maps[i].cpu().numpy(), mref) <= 1e-3
        for g in envs:
            g.close()
    finally:
        pool.terminate()
        pool.join()
