"""Seeded parity cases on the workloads the benchmark runs, with the FP64
oracle's run of each (test infrastructure: only the GPU parity tests import
this module; it imports the oracle and the input generators, never the CUDA
library, so it can run in spawned worker processes beside the GPU tests).

Cases (Algorithm 2's step, dynamic dt = 1/60 s unless stated):
  pad-sphere / pad-cylinder / pad-box  graded GelSight-like pad (~3.4k tets),
      each indenter family, full depth reached in 4 steps with tangential
      slip; 3 steps are run.  (Some box seeds are bistable: a filleted edge
      sliding over gel vertices has two nearby local minima, and FP32 and
      FP64 arithmetic can settle in different ones; seed 5 is not.)
  bench-59k   the 59,220-tet bench env itself (its first load step).
  close-pairs small pad of 1 mm elements under a 3 mm sphere with a barrier
      stiffness of 1 N/m, so that contact pairs settle below 1e-2 dhat
      (quasi-static).
  parallel-edges small pad under a cylinder lying along the pad's x edges
      (gel and indenter edges exactly parallel: the edge-edge mollifier is
      active), quasi-static.
  pad-friction the pad-sphere case with friction ratio 0.5 and velocity
      threshold 0.01 m/s (Sec. III-B), its slip doubled.
  dual-layer  a 9DTact-like block with a soft top layer over a stiff base
      (per-tet material), the first of 4 dynamic steps.
"""
import copy
import math

import numpy as np

from synth import indenters, meshes, workloads

CASES = ["pad-sphere", "pad-cylinder", "pad-box", "bench-59k", "close-pairs", "parallel-edges", "pad-friction",
         "dual-layer"]
STEPS = {"pad-sphere": 3, "pad-cylinder": 3, "pad-box": 3, "bench-59k": 1, "close-pairs": 1, "parallel-edges": 2,
         "pad-friction": 3, "dual-layer": 1}


def _pose(tx, ty, tz):
    return dict(R=np.eye(3), t=np.array([tx, ty, tz], dtype=np.float64))


def build_case(name):
    """The environment dictionary of a case (inputs only)."""
    if name == "pad-friction":
        env = copy.deepcopy(workloads.gelsight_env(3, steps=4, target_tets=4000, grid_hw=(60, 80)))
        t0 = env["start_pose"]["t"]
        for p in env["poses"]:
            p["t"][:2] = t0[:2] + 2.0 * (p["t"][:2] - t0[:2])
        env["opts"]["friction_mu"] = 0.5
        env["opts"]["friction_eps_v"] = 0.01
        return env
    if name.startswith("pad-"):
        seed = {"pad-sphere": 3, "pad-cylinder": 0, "pad-box": 5}[name]
        env = workloads.gelsight_env(seed, steps=4, target_tets=4000, grid_hw=(60, 80))
        assert env["kind"] == name[4:]
        return env
    if name == "dual-layer":
        return workloads.dual_layer_env(2, target_tets=4000, steps=4)
    if name == "bench-59k":
        return workloads.gelsight_env(0, mesh=meshes.graded_pad())
    if name == "close-pairs":
        # a 3 mm sphere pressed 0.05 mm into a pad of 1 mm elements with kappa =
        # 1 N/m: the barrier carries the load at pair distances of ~3e-3 dhat
        # (about 90 CCD-limited substeps)
        env = copy.deepcopy(workloads.small_env(8, nx=8, ny=8, nz=2, steps=1, step_depth=0.05e-3, radius=3e-3,
                                                level=4))
        env["opts"]["kappa"] = 1.0
        return env
    if name == "parallel-edges":
        Lx, Ly, Lz, dhat = 8e-3, 8e-3, 2e-3, 0.05e-3
        X, T = meshes.box(4, 4, 2, Lx, Ly, Lz)
        R = 1.5e-3
        # 20 segments around the axis, so that one generator line is the lowest
        V, F = indenters.cylinder(R, 12e-3, 2 * math.pi * R / 20 * 1.0001)
        low = indenters.lowest_z(V)
        # the cylinder's lowest generator line lies over the grid line y = Ly/2
        cx, cy = Lx / 2, Ly / 2
        start = _pose(cx, cy, Lz + dhat - low)
        poses = [_pose(cx, cy, Lz - 0.04e-3 * k - low) for k in (1, 2)]
        grid = dict(axis_u=0, axis_v=1, origin=(0.0, 0.0), pixel=(Lx / 16, Ly / 16), H=16, W=16)
        opts = dict(dhat=dhat, kappa=0.0, dt=0.0, newton_rtol=1e-6, newton_max=1024, pcg_max=1000,
                    precision="fp64", contact_axis=-1)
        return dict(name="parallel-edges", X=X, tets=T, material=dict(workloads.MATERIAL),
                    fixed=np.nonzero(X[:, 2] == 0.0)[0].astype(np.int32), ind_V=V, ind_F=F, start_pose=start,
                    poses=poses, grid=grid, opts=opts, depth=0.08e-3, kind="cylinder")
    raise KeyError(name)


def run_case(name):
    """Step the oracle through the case's poses; returns the Scene (picklable)."""
    from oracle.sim import Scene
    env = build_case(name)
    sc = Scene(env)
    for k in range(STEPS[name]):
        sc.step(env["poses"][k])
    return sc


def min_pair_distance(sc, x):
    return sc.min_distance(x, sc.indenter(sc.pose))


def parallel_ee_pairs(sc, x):
    """Edge-edge pairs within dhat whose mollifier is active (|e0 x e1|^2
    below eps_x = 1e-3 |e0|^2 |e1|^2 of the rest lengths)."""
    from oracle import geometry as geo
    Y = sc.indenter(sc.pose)
    gi, ii = sc.candidates(x, Y)["ee"]
    if len(gi) == 0:
        return 0
    pts = sc.pair_points("ee", gi, ii, x, Y)
    d2, _ = geo.distance_sq(pts, "ee")
    c, _, _ = geo.cross_sq(pts)
    act = (np.sqrt(d2) < sc.dhat) & (c < sc.eps_x(gi, ii))
    return int(act.sum())
