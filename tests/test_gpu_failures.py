"""Failure paths of the C ABI made on the host (no GPU fault): a device
allocator that runs out, the Newton iteration cap (Sec. III-B's 1024 is the
method's only stated failure bound; here it is set to 1), PCG caps, and
per-env PCG caps inside one batched launch."""
import copy
import ctypes

import numpy as np
import pytest

from gpu_util import rel_fro
from oracle.sim import NewtonMaxIter, Scene
from synth import workloads

pytestmark = pytest.mark.gpu


class LimitedAllocator:
    """tc_allocator over the PyTorch caching allocator that refuses every
    request after the first `limit` ones and records what is still held."""

    def __init__(self, limit):
        import torch
        from paper_2606_20426_gb300 import tacauchy as tcm
        self.limit, self.n, self.refused, self.live = limit, 0, 0, set()

        def alloc(ctx, nbytes, stream):
            if self.n >= self.limit:
                self.refused += 1
                return None
            self.n += 1
            p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            self.live.add(int(p))
            return p

        def release(ctx, ptr, nbytes, stream):
            self.live.discard(int(ptr))
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a, self._r = tcm.ALLOC_FN(alloc), tcm.RELEASE_FN(release)
        self.struct = tcm.Allocator(self._a, self._r, None)


def test_allocator_running_out_gives_oom_and_releases_everything():
    from paper_2606_20426_gb300 import Env, TcError
    env = workloads.small_env(0, steps=1)
    for limit in (0, 3, 25):
        a = LimitedAllocator(limit)
        with pytest.raises(TcError) as ei:
            Env(env, allocator=a)
        assert ei.value.code == 9  # TC_ERR_OOM
        assert a.refused >= 1 and a.n == limit and not a.live  # every block it handed out came back
    # the library and the device are fine afterwards
    g = Env(env)
    g.step(env["poses"][0])
    g.close()


def _with_opts(env, **kw):
    env = copy.deepcopy(env)
    env["opts"].update(kw)
    return env


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_newton_cap_fails_the_step_and_restores_the_env(precision):
    from paper_2606_20426_gb300 import Env, TcError
    env = _with_opts(workloads.small_env(1, steps=1), newton_max=1)
    with pytest.raises(NewtonMaxIter):   # the oracle with the same cap
        Scene(env).step(env["poses"][0])
    g = Env(env, precision=precision)
    x0 = g.positions()
    with pytest.raises(TcError) as ei:
        g.step(env["poses"][0])
    assert ei.value.code == 4  # TC_ERR_NEWTON_MAXITER
    assert np.array_equal(g.positions(), x0)
    # the indenter is back at its start pose: stepping to it needs no iteration
    g.step(env["start_pose"])
    assert np.array_equal(g.positions(), x0)
    g.close()


@pytest.mark.parametrize("pcg_max", [1, 4])
def test_pcg_cap_is_counted_and_the_step_still_converges(pcg_max):
    """A capped PCG solve is a descent direction, so Newton goes on with it;
    the converged state is the oracle's."""
    from paper_2606_20426_gb300 import Env
    env = _with_opts(workloads.small_env(2, steps=1), pcg_max=pcg_max)
    g = Env(env, precision="fp64")
    g.step(env["poses"][0])
    ref = Scene(env)
    ref.step(env["poses"][0])
    info = g.get_info()
    assert info["pcg_capped"] > 0
    assert info["pcg_iters"] <= pcg_max * info["newton_iters"]
    x = g.positions()
    assert np.abs(x - ref.x).max() <= 1e-3 * env["depth"]
    f, fr = g.contact_force(), ref.contact_force()
    assert np.linalg.norm(f - fr) <= 5e-3 * np.linalg.norm(fr)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_keeps_each_envs_own_pcg_cap(precision):
    """Envs with different pcg_max in one tc_step_batch give, bit for bit,
    what each gives alone (each stops at its own cap inside the shared
    cluster launch)."""
    from paper_2606_20426_gb300 import Env, step_batch
    envs = [_with_opts(workloads.small_env(3, steps=2), pcg_max=3),
            _with_opts(workloads.small_env(4, steps=2), pcg_max=1000),
            _with_opts(workloads.small_env(5, steps=2), pcg_max=7)]
    alone = [Env(e, precision=precision) for e in envs]
    batch = [Env(e, precision=precision) for e in envs]
    for k in range(2):
        for g, e in zip(alone, envs):
            g.step(e["poses"][k])
        assert step_batch(batch, [e["poses"][k] for e in envs]) == [0, 0, 0]
    for a, b in zip(alone, batch):
        assert np.array_equal(a.positions(), b.positions())
        ia, ib = a.get_info(), b.get_info()
        assert (ia["pcg_iters"], ia["pcg_capped"], ia["newton_iters"]) == (ib["pcg_iters"], ib["pcg_capped"],
                                                                           ib["newton_iters"])
    assert alone[0].get_info()["pcg_capped"] > 0 and alone[1].get_info()["pcg_capped"] == 0
    for g in alone + batch:
        g.close()
