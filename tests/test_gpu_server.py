"""Step server (continuous batching): requests that arrive at seeded Poisson
times from envs of different sizes and precisions, and join while others are
on the GPU, give results bit-identical to the same env stepped alone; the
stress and pressure-map buffers given at submit hold tc_stress /
tc_pressure_map of the result; admission by slots and HBM footprint; an env
with a pending request is refused by tc_step; waits time out instead of
hanging."""
import threading
import time

import numpy as np
import pytest

from synth import workloads

pytestmark = pytest.mark.gpu


def _scenes():
    return [("fp64", workloads.small_env(0)), ("fp32", workloads.small_env(5)),
            ("fp64", workloads.pad_env(1, steps=2)), ("fp32", workloads.small_env(4, dt=1.0 / 60.0)),
            ("fp32", workloads.pad_env(2, steps=2))]


def _alone(prec, scene, nsteps):
    from paper_2606_20426_gb300 import Env
    g = Env(scene, precision=prec)
    for k in range(nsteps):
        g.step(scene["poses"][k])
    return g


def _outputs(torch, g):
    sig = torch.empty((6, g.info["nt"]), dtype=torch.float32, device="cuda")
    m = torch.empty((g.info["H"], g.info["W"]), dtype=torch.float32, device="cuda")
    k = torch.empty((g.info["H"], g.info["W"]), dtype=torch.uint8, device="cuda")
    return sig, m, k


def test_server_mix_equals_alone():
    import torch
    from paper_2606_20426_gb300 import Env, Server
    scenes = _scenes()
    nsteps = 2
    envs = [Env(s, precision=p) for p, s in scenes]
    outs = [_outputs(torch, g) for g in envs]
    srv = Server(hbm_budget_bytes=1 << 40, max_slots=64, workers=2)
    delays = np.random.default_rng(3).exponential(0.01, size=len(envs))
    results = {}

    def client(i):
        # each env submits its next pose once the previous one is done; the
        # first submission arrives after a seeded exponential delay
        time.sleep(float(delays[i]) * (i + 1))
        for k in range(nsteps):
            t = srv.submit(envs[i], scenes[i][1]["poses"][k], *outs[i])
            r = srv.wait(t, timeout_s=300.0)
            assert r is not None
            results[(i, k)] = r

    th = [threading.Thread(target=client, args=(i,)) for i in range(len(envs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    info = srv.info()
    srv.close()
    assert all(r["status"] == 0 for r in results.values()), results
    assert info["completed"] == len(envs) * nsteps
    assert info["peak_inflight"] >= 2  # requests really overlapped on the device
    torch.cuda.synchronize()
    for (p, s), g, (sig, m, k) in zip(scenes, envs, outs):
        a = _alone(p, s, nsteps)
        assert np.array_equal(g.positions(), a.positions())
        assert np.array_equal(sig.cpu().numpy(), a.stress().cpu().numpy())
        am, ak = a.pressure_map()
        assert np.array_equal(m.cpu().numpy(), am.cpu().numpy())
        assert np.array_equal(k.cpu().numpy(), ak.cpu().numpy())
        assert g.get_info()["steps"] == nsteps
        a.close()
        g.close()


def test_server_one_slot_and_budget():
    from paper_2606_20426_gb300 import Env, Server
    s0, s1 = workloads.small_env(0), workloads.small_env(5)
    g0, g1 = Env(s0), Env(s1)
    srv = Server(hbm_budget_bytes=1 << 40, max_slots=1)
    t0 = srv.submit(g0, s0["poses"][0])
    t1 = srv.submit(g1, s1["poses"][0])
    r0, r1 = srv.wait(t0, 300.0), srv.wait(t1, 300.0)
    assert r0["status"] == 0 and r1["status"] == 0
    assert srv.info()["peak_inflight"] == 1
    srv.close()
    for g, s in ((g0, s0), (g1, s1)):
        a = _alone("fp64", s, 1)
        assert np.array_equal(g.positions(), a.positions())
        a.close()
    # a budget below the env's footprint: the request is refused at admission
    tiny = Server(hbm_budget_bytes=1024, max_slots=4)
    x = g0.positions()
    r = tiny.wait(tiny.submit(g0, s0["poses"][1]), 60.0)
    assert r["status"] == 10
    assert np.array_equal(g0.positions(), x)
    tiny.close()
    g0.close()
    g1.close()


def test_pending_env_refused_and_wait_timeout():
    from paper_2606_20426_gb300 import Env, Server, TcError
    s = workloads.pad_env(1, steps=2)
    g = Env(s)
    srv = Server(hbm_budget_bytes=1 << 40, max_slots=4)
    t = srv.submit(g, s["poses"][0])
    # the pad's step takes far longer than these host calls
    assert srv.wait(t, timeout_s=0.0) is None
    with pytest.raises(TcError) as ei:
        g.step(s["poses"][0])
    assert ei.value.code == 1
    r = srv.wait(t, timeout_s=300.0)
    assert r["status"] == 0 and r["latency_us"] > 0 and r["rounds"] >= 1
    with pytest.raises(TcError):
        srv.poll(t)  # the ticket was released
    bad = dict(s["poses"][1])
    bad["t"] = np.array([np.inf, 0.0, 0.0])
    with pytest.raises(TcError) as ei:
        srv.submit(g, bad)
    assert ei.value.code == 7
    srv.close()
    g.step(s["poses"][1])  # the env is free again
    g.close()


def test_budget_meters_working_sets_and_evicts_idle_ones():
    """A budget that holds the working sets of two of four envs: requests of
    all four (round robin, three steps each) complete with the results of
    the same envs stepped alone, bit for bit; the server released idle
    working sets to make room (evictions > 0), never holds more than the
    budget once the requests are done, and an evicted env steps again on its
    own (its working set comes back)."""
    from paper_2606_20426_gb300 import Env, Server
    cfgs = [workloads.small_env(s, steps=3) for s in (0, 1, 2, 3)]
    alone = [Env(c) for c in cfgs]
    served = [Env(c) for c in cfgs]
    wb = served[0].get_info()["working_bytes"]
    assert wb > 0 and all(e.get_info()["working_resident"] == 1 for e in served)
    budget = int(2.5 * max(e.get_info()["working_bytes"] for e in served))
    srv = Server(hbm_budget_bytes=budget, max_slots=2, workers=2)
    for k in range(3):
        tickets = [srv.submit(e, c["poses"][k]) for e, c in zip(served, cfgs)]
        for t in tickets:
            r = srv.wait(t, 120.0)
            assert r is not None and r["status"] == 0
        for e, c in zip(alone, cfgs):
            e.step(c["poses"][k])
    st = srv.info()
    assert st["evictions"] > 0 and st["known_envs"] == 4
    assert st["inflight_bytes"] <= budget
    resident = sum(e.get_info()["working_resident"] for e in served)
    assert 1 <= resident <= 2
    for a, b in zip(alone, served):
        assert np.array_equal(a.positions(), b.positions())
    # an evicted env is used directly again
    idle = [e for e in served if e.get_info()["working_resident"] == 0][0]
    idle.step(cfgs[served.index(idle)]["poses"][2])
    assert idle.get_info()["working_resident"] == 1
    served[3].close()
    assert srv.info()["known_envs"] == 3
    srv.close()
    for e in alone + served[:3]:
        e.close()
