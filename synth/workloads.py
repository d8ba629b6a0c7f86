"""Seeded synthetic environments: gel mesh + material + fixed set + rigid
indenter + pose schedule + pixel grid + solver options.

Environment dictionaries hold plain numpy arrays and numbers; both the oracle
and the CUDA binding consume them.  Recipes (sizes in metres):

* ``pad_env``      - 20x20x4 mm box, 10x10x3 hexes (1,800 tets, 484 verts),
                     E = 0.3 MPa, nu = 0.45, rho = 1100, bottom fixed, sphere
                     R = 5 mm (icosphere, edge <= 0.25 mm) centred at
                     (10, 10) mm +- U[-1, 1] mm; quasi-static, dhat = 0.05 mm;
                     starts dhat above the top and goes down 0.05 mm per step
                     for 10 steps; 32x32 pixel grid over the top face.
* ``gelsight_env`` - graded 18x24x4 mm pad (~60k tets) pressed by a seeded
                     sphere (R~U[2,6] mm), cylinder (R~U[1,3] mm, axis in the
                     pad plane at a random angle) or 4 mm box with a 0.2 mm
                     fillet, to depth U[0.2, 1.0] mm with tangential slip
                     U[0, 0.5] mm over 20 dynamic steps at dt = 1/60 s; 240x320
                     grid (0.075 mm pixels).
* ``small_env``    - a few hundred tets, for tests that run the oracle's full
                     Newton solve in seconds.
* ``sensor_env``   - the same kind of indentation on a pad, DIGIT-like dome or
                     9DTact-like block of a given size; ``mixed_envs`` draws an
                     uneven batch of the three families.
"""
import math
import numpy as np

from . import meshes, indenters
from .rng import SplitMix64

MATERIAL = dict(E=3.0e5, nu=0.45, density=1100.0)


def _opts(dhat, dt, precision):
    return dict(dhat=dhat, kappa=0.0, dt=dt, newton_rtol=1e-6, newton_max=1024,
                pcg_max=1000, precision=precision, contact_axis=-1)


def _pose(tx, ty, tz, yaw=0.0):
    c, s = math.cos(yaw), math.sin(yaw)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return dict(R=R, t=np.array([tx, ty, tz], dtype=np.float64))


def _fixed_bottom(X):
    return np.nonzero(X[:, 2] == 0.0)[0].astype(np.int32)


def icosphere_level_for(radius, edge):
    return max(1, int(math.ceil(math.log2(1.06 * radius / edge))))


def pad_env(seed, steps=10, step_depth=0.05e-3, nx=10, ny=10, nz=3,
            size=(20e-3, 20e-3, 4e-3), radius=5e-3, edge=0.25e-3, dhat=0.05e-3,
            grid_hw=(32, 32), precision="fp64", jitter=1e-3):
    rng = SplitMix64(seed)
    Lx, Ly, Lz = size
    X, T = meshes.box(nx, ny, nz, Lx, Ly, Lz)
    V, F = indenters.icosphere(radius, icosphere_level_for(radius, edge))
    cx = Lx / 2 + rng.uniform(-jitter, jitter)
    cy = Ly / 2 + rng.uniform(-jitter, jitter)
    low = indenters.lowest_z(V)
    start = _pose(cx, cy, Lz + dhat - low)
    poses = [_pose(cx, cy, Lz - step_depth * k - low) for k in range(1, steps + 1)]
    H, W = grid_hw
    grid = dict(axis_u=0, axis_v=1, origin=(0.0, 0.0), pixel=(Lx / W, Ly / H), H=H, W=W)
    return dict(name=f"pad{nx}x{ny}x{nz}-seed{seed}", X=X, tets=T, material=dict(MATERIAL),
                fixed=_fixed_bottom(X), ind_V=V, ind_F=F, start_pose=start, poses=poses,
                grid=grid, opts=_opts(dhat, 0.0, precision), depth=step_depth * steps)


def small_env(seed, nx=4, ny=4, nz=2, size=(8e-3, 8e-3, 2e-3), radius=3e-3, level=3,
              steps=2, step_depth=0.05e-3, dhat=0.05e-3, dt=0.0, precision="fp64"):
    rng = SplitMix64(seed)
    Lx, Ly, Lz = size
    X, T = meshes.box(nx, ny, nz, Lx, Ly, Lz)
    V, F = indenters.icosphere(radius, level)
    cx = Lx / 2 + rng.uniform(-0.5e-3, 0.5e-3)
    cy = Ly / 2 + rng.uniform(-0.5e-3, 0.5e-3)
    low = indenters.lowest_z(V)
    start = _pose(cx, cy, Lz + dhat - low)
    poses = [_pose(cx, cy, Lz - step_depth * k - low) for k in range(1, steps + 1)]
    grid = dict(axis_u=0, axis_v=1, origin=(0.0, 0.0), pixel=(Lx / 16, Ly / 16), H=16, W=16)
    return dict(name=f"small{nx}x{ny}x{nz}-seed{seed}", X=X, tets=T, material=dict(MATERIAL),
                fixed=_fixed_bottom(X), ind_V=V, ind_F=F, start_pose=start, poses=poses,
                grid=grid, opts=_opts(dhat, dt, precision), depth=step_depth * steps)


def gelsight_indenter(rng, edge=0.25e-3):
    """Seeded indenter for the GelSight-like pad: (kind, V, F, yaw)."""
    kind = ("sphere", "cylinder", "box")[rng.integers(3)]
    if kind == "sphere":
        r = rng.uniform(2e-3, 6e-3)
        V, F = indenters.icosphere(r, icosphere_level_for(r, edge))
        yaw = 0.0
    elif kind == "cylinder":
        r = rng.uniform(1e-3, 3e-3)
        V, F = indenters.cylinder(r, 30e-3, edge)
        yaw = rng.uniform(0.0, math.pi)
    else:
        V, F = indenters.rounded_box((2e-3, 2e-3, 2e-3), 0.2e-3, edge)
        yaw = rng.uniform(0.0, 0.5 * math.pi)
    return kind, V, F, yaw


def gelsight_env(seed, steps=20, target_tets=60000, dhat=0.05e-3, dt=1.0 / 60.0,
                 precision="fp32", grid_hw=(240, 320), mesh=None):
    rng = SplitMix64(seed)
    Lx, Ly, Lz = 18e-3, 24e-3, 4e-3
    X, T = mesh if mesh is not None else meshes.graded_pad(Lx, Ly, Lz, target_tets=target_tets)
    kind, V, F, yaw = gelsight_indenter(rng)
    cx = Lx / 2 + rng.uniform(-2e-3, 2e-3)
    cy = Ly / 2 + rng.uniform(-2e-3, 2e-3)
    depth = rng.uniform(0.2e-3, 1.0e-3)
    slip = rng.uniform(0.0, 0.5e-3)
    phi = rng.uniform(0.0, 2 * math.pi)
    # lowest point of the yawed indenter (yaw is about z, so z extents are kept)
    low = indenters.lowest_z(V)
    z0 = Lz + dhat - low
    start = _pose(cx, cy, z0, yaw)
    poses = []
    for k in range(1, steps + 1):
        f = k / steps
        poses.append(_pose(cx + f * slip * math.cos(phi), cy + f * slip * math.sin(phi),
                           z0 - f * (dhat + depth), yaw))
    H, W = grid_hw
    # rows along x (the 18 mm side), columns along y (the 24 mm side)
    grid = dict(axis_u=1, axis_v=0, origin=(0.0, 0.0), pixel=(Ly / W, Lx / H), H=H, W=W)
    return dict(name=f"gelsight-{kind}-seed{seed}", X=X, tets=T, material=dict(MATERIAL),
                fixed=_fixed_bottom(X), ind_V=V, ind_F=F, start_pose=start, poses=poses,
                grid=grid, opts=_opts(dhat, dt, precision), depth=depth, kind=kind)


def _grid_over(Lx, Ly, pixel):
    """Pixel grid over the x-y extent: rows along x, columns along y."""
    H, W = max(1, int(round(Lx / pixel))), max(1, int(round(Ly / pixel)))
    return dict(axis_u=1, axis_v=0, origin=(0.0, 0.0), pixel=(Ly / W, Lx / H), H=H, W=W)


def sensor_mesh(sensor, target_tets):
    """Mesh of a sensor family scaled to about target_tets tets:
    'pad'   graded 18x24x4 mm pad (GelSight-Mini-like),
    'dome'  20x16 mm base with a 1.5 mm slab and a spherical cap of radius
            30 mm and height 3 mm clipped to the base (DIGIT-like),
    'block' 30x30x5 mm block (9DTact-like), uniform hexes split 6 ways."""
    if sensor == "pad":
        return meshes.graded_pad(target_tets=target_tets), (18e-3, 24e-3)
    if sensor == "dome":
        nz = 6
        s = math.sqrt(target_tets / (6.0 * nz * 20 * 16))
        nx, ny = max(4, int(round(20 * s))), max(4, int(round(16 * s)))
        return meshes.dome(nx=nx, ny=ny, nz=nz), (20e-3, 16e-3)
    if sensor == "block":
        nz = max(2, int(round((target_tets / 6.0 / 36.0) ** (1.0 / 3.0))))
        n = max(4, int(round(math.sqrt(target_tets / (6.0 * nz)))))
        return meshes.block(nx=n, ny=n, nz=nz), (30e-3, 30e-3)
    raise ValueError(sensor)


def sensor_env(seed, sensor="pad", target_tets=20000, steps=20, dhat=0.05e-3, dt=1.0 / 60.0,
               precision="fp32", pixel=0.1e-3, mesh=None):
    """A GelSight-style indentation (seeded sphere / cylinder / filleted box,
    depth U[0.2, 1.0] mm, slip U[0, 0.5] mm over `steps` dynamic steps) on a
    pad, dome or block sensor of about target_tets tets; the indenter starts
    dhat above the highest gel point near the sensor centre.  mesh: a
    ((X, T), (Lx, Ly)) from sensor_mesh to reuse."""
    rng = SplitMix64(seed)
    (X, T), (Lx, Ly) = mesh if mesh is not None else sensor_mesh(sensor, target_tets)
    kind, V, F, yaw = gelsight_indenter(rng)
    cx = Lx / 2 + rng.uniform(-1e-3, 1e-3)
    cy = Ly / 2 + rng.uniform(-1e-3, 1e-3)
    depth = rng.uniform(0.2e-3, 1.0e-3)
    slip = rng.uniform(0.0, 0.5e-3)
    phi = rng.uniform(0.0, 2 * math.pi)
    top = float(X[:, 2].max())
    z0 = top + dhat - indenters.lowest_z(V)
    start = _pose(cx, cy, z0, yaw)
    poses = []
    for k in range(1, steps + 1):
        f = k / steps
        poses.append(_pose(cx + f * slip * math.cos(phi), cy + f * slip * math.sin(phi),
                           z0 - f * (dhat + depth), yaw))
    return dict(name=f"{sensor}-{kind}-seed{seed}", X=X, tets=T, material=dict(MATERIAL),
                fixed=_fixed_bottom(X), ind_V=V, ind_F=F, start_pose=start, poses=poses,
                grid=_grid_over(Lx, Ly, pixel), opts=_opts(dhat, dt, precision), depth=depth, kind=kind,
                sensor=sensor)


def mixed_envs(seed, n_per_family=20, pads=(5000, 60000), domes=(8000, 40000), blocks=(10000, 80000),
               steps=20, precision="fp32"):
    """Uneven batch of pads, domes and blocks, sizes log-uniform in the given
    tet ranges, each with its own seeded indenter."""
    rng = SplitMix64(seed)
    out = []
    for fam, (lo, hi) in (("pad", pads), ("dome", domes), ("block", blocks)):
        for i in range(n_per_family):
            nt = int(math.exp(rng.uniform(math.log(lo), math.log(hi))))
            out.append(sensor_env(seed * 1000 + len(out), fam, nt, steps=steps, precision=precision))
    return out


DUAL_LAYER = dict(top_thickness=1.5e-3, E_top=0.3e6, E_base=1.2e6, nu=0.45)


def dual_layer_material(X, T, top_thickness=DUAL_LAYER["top_thickness"], E_top=DUAL_LAYER["E_top"],
                        E_base=DUAL_LAYER["E_base"], nu=DUAL_LAYER["nu"]):
    """(E, nu) per tet of a two-layer gel: tets whose centroid lies within
    top_thickness of the top face take E_top, the rest E_base (the paper names
    a dual-layer 9DTact pad without giving its values; these are the stand-in
    values of this build)."""
    ztop = X[:, 2].max()
    zc = X[T].mean(axis=1)[:, 2]
    E = np.where(zc >= ztop - top_thickness, E_top, E_base)
    return np.stack([E, np.full(len(T), nu)], axis=1)


def dual_layer_env(seed, target_tets=20000, steps=20, precision="fp32", mesh=None):
    """The 9DTact-like block of sensor_env with a soft top layer over a stiff
    base (per-tet material)."""
    env = sensor_env(seed, "block", target_tets, steps=steps, precision=precision, mesh=mesh)
    env["material"]["per_tet"] = dual_layer_material(env["X"], env["tets"])
    env["name"] = env["name"].replace("block", "dual-block")
    return env


def scale_envs(seed, n=1024, target_tets=20000, steps=20, precision="fp32"):
    """n environments of about target_tets tets, pads and domes alternating
    (one mesh per family, shared), each with its own seeded indenter."""
    meshes_ = {fam: sensor_mesh(fam, target_tets) for fam in ("pad", "dome")}
    return [sensor_env(seed * 100000 + i, fam, target_tets, steps=steps, precision=precision, mesh=meshes_[fam])
            for i, fam in zip(range(n), ("pad", "dome") * n)]


def sphere_cluster(radius=3e-3, spacing=7e-3, edge=0.25e-3):
    """Three icospheres of the same radius at the corners of an equilateral
    triangle (side `spacing`) in the z = 0 plane, as one rigid surface."""
    V1, F1 = indenters.icosphere(radius, icosphere_level_for(radius, edge))
    Vs, Fs = [], []
    for k in range(3):
        a = 2 * math.pi * k / 3
        c = spacing / math.sqrt(3.0) * np.array([math.cos(a), math.sin(a), 0.0])
        Fs.append(F1 + len(V1) * k)
        Vs.append(V1 + c)
    return np.concatenate(Vs), np.concatenate(Fs).astype(np.int32)


def big_pad_env(target_tets=2_000_000, depth=0.8e-3, steps=20, dhat=0.05e-3, dt=1.0 / 60.0, precision="fp32",
                grid_hw=(240, 320)):
    """A GelSight-like 18x24x4 mm pad refined to about target_tets tets under
    a cluster of three R = 3 mm spheres pressed to `depth` over `steps`
    dynamic steps."""
    Lx, Ly, Lz = 18e-3, 24e-3, 4e-3
    X, T = meshes.graded_pad(Lx, Ly, Lz, target_tets=target_tets)
    V, F = sphere_cluster()
    cx, cy = Lx / 2, Ly / 2
    z0 = Lz + dhat - indenters.lowest_z(V)
    start = _pose(cx, cy, z0)
    poses = [_pose(cx, cy, z0 - (k / steps) * (dhat + depth)) for k in range(1, steps + 1)]
    H, W = grid_hw
    grid = dict(axis_u=1, axis_v=0, origin=(0.0, 0.0), pixel=(Ly / W, Lx / H), H=H, W=W)
    return dict(name=f"bigpad-{len(T)}", X=X, tets=T, material=dict(MATERIAL), fixed=_fixed_bottom(X), ind_V=V,
                ind_F=F, start_pose=start, poses=poses, grid=grid, opts=_opts(dhat, dt, precision), depth=depth,
                kind="sphere-cluster")


def hertz_env(nu=0.3, radius=5e-3, depth=0.25e-3, steps=5, dhat=0.01e-3, precision="fp32"):
    """Frictionless sphere pressed quasi-statically into a 20 x 20 x 10 mm
    block (bottom fixed) refined to 0.12 mm under the contact: the setting
    of the Hertz force-indentation law F = 4/3 E* sqrt(R) delta^(3/2),
    E* = E / (1 - nu^2), for a contact radius sqrt(R delta) << block size."""
    X, T = meshes.hertz_block()
    L = 20e-3
    top = float(X[:, 2].max())
    V, F = indenters.icosphere(radius, icosphere_level_for(radius, 0.1e-3))
    z0 = top + dhat - indenters.lowest_z(V)
    start = _pose(L / 2, L / 2, z0)
    poses = [_pose(L / 2, L / 2, z0 - (dhat + depth) * k / steps) for k in range(1, steps + 1)]
    mat = dict(MATERIAL)
    mat["nu"] = nu
    return dict(name=f"hertz-nu{nu}", X=X, tets=T, material=mat, fixed=_fixed_bottom(X), ind_V=V, ind_F=F,
                start_pose=start, poses=poses, grid=None, opts=_opts(dhat, 0.0, precision), depth=depth,
                radius=radius, top=top)


def splitmix64_array(seed, n):
    """n outputs of splitmix64 as a counter-based generator: output i is the
    mix of state seed + (i+1)*gamma (vectorised, uint64 wrap-around)."""
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.arange(1, n + 1, dtype=np.uint64) * g)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def random_deformation_gradients(seed, n, max_norm=0.3):
    """F = I + S per tet, S symmetric with Gaussian entries scaled to
    ||S||_F = max_norm * U[0,1]; float64 (n, 3, 3).  Eigenvalues of F stay
    in [1 - max_norm, 1 + max_norm], so F is SPD and det F > 0."""
    z = splitmix64_array(seed, 8 * n).reshape(n, 8)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    u1 = 1.0 - u[:, 0:3]
    u2 = u[:, 3:6]
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)], axis=1)
    S = np.empty((n, 3, 3))
    S[:, 0, 0], S[:, 1, 1], S[:, 2, 2] = g[:, 0], g[:, 1], g[:, 2]
    S[:, 0, 1] = S[:, 1, 0] = g[:, 3]
    S[:, 1, 2] = S[:, 2, 1] = g[:, 4]
    S[:, 0, 2] = S[:, 2, 0] = g[:, 5]
    nrm = np.sqrt(np.einsum("nij,nij->n", S, S))
    scale = max_norm * u[:, 6] / np.maximum(nrm, 1e-300)
    return np.eye(3)[None] + S * scale[:, None, None]
