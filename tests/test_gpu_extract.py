"""GPU parity of scene setup and stress extraction (rows a0, a10-a13) against
the FP64 oracle, through the C ABI.

* integer outputs (boundary faces, parents, contact faces, pixel binning) are
  bit-exact, and so are the FP32 barycentric weights (same FP64 arithmetic,
  rounded once);
* given identical positions, sigma matches to relative Frobenius <= 1e-4 and
  the pressure map to relative L2 <= 1e-3 (FP64 and mixed FP32 modes).
"""
import copy

import numpy as np
import pytest

from gpu_util import rel_fro
from oracle import material as mat
from oracle.sim import Scene
from synth import workloads

pytestmark = pytest.mark.gpu


def _gpu_env(env, precision="fp64"):
    from paper_2606_20426_gb300 import Env
    return Env(env, precision=precision)


def _smooth_positions(X, amp=1.5e-4, seed=0):
    """Rest positions plus a smooth, seeded displacement field (an input)."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(100, 400, size=(3, 3))
    ph = rng.uniform(0, 2 * np.pi, size=(3, 3))
    u = np.zeros_like(X)
    for i in range(3):
        for j in range(3):
            u[:, i] += amp * np.sin(k[i, j] * X[:, j] + ph[i, j]) / 3
    return X + u


ENVS = {
    "pad1800": lambda: workloads.pad_env(0),
    "small": lambda: workloads.small_env(3),
    "gelsight60k": lambda: workloads.gelsight_env(0),
}


@pytest.fixture(scope="module", params=list(ENVS))
def pair(request):
    env = ENVS[request.param]()
    return env, Scene(env)


def test_setup_tables_bit_exact(pair):
    env, ref = pair
    g = _gpu_env(env)
    f, p = g.boundary_faces()
    assert np.array_equal(f, ref.faces) and np.array_equal(p, ref.parent)
    cf, cp = g.surface_faces()
    assert np.array_equal(cf, ref.cfaces) and np.array_equal(cp, ref.cparent)
    pf, pw = g.pixel_table()
    assert np.array_equal(pf, ref.pix_face)
    assert np.array_equal(pw.view(np.uint32), ref.pix_w.view(np.uint32))
    inf = g.info
    assert inf["nvc"] == len(ref.cverts) and inf["nec"] == len(ref.cedges)
    assert inf["kappa"] == pytest.approx(ref.kappa, rel=1e-12)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stress_traction_map_given_positions(pair, precision):
    env, ref = pair
    g = _gpu_env(env, precision)
    x = _smooth_positions(ref.X)
    g.set_positions(x)
    xg = g.positions()  # the positions the GPU holds (FP32 mode rounds u once)
    sig = g.stress().cpu().numpy().T
    sref = ref.stress(xg)
    assert rel_fro(sig, sref) <= 1e-4
    # traction / pressure / tangential traction on the contact faces
    t, p, tt = (a.cpu().numpy() for a in g.traction())
    tr, pr, ttr = ref.traction(xg)
    assert rel_fro(t.T, tr) <= 1e-4
    assert rel_fro(p, pr) <= 1e-4
    assert rel_fro(tt.T, ttr) <= 1e-3
    m, mask = g.pressure_map()
    mref, maskref = ref.pressure_map(x=xg)
    assert np.array_equal(mask.cpu().numpy(), maskref)
    assert rel_fro(m.cpu().numpy(), mref) <= 1e-3
    g.close()


def test_rest_state_is_zero(pair):
    env, _ = pair
    g = _gpu_env(env, "fp32")
    sig = g.stress().cpu().numpy()
    assert np.abs(sig).max() == 0.0
    m, _ = g.pressure_map()
    assert np.abs(m.cpu().numpy()).max() == 0.0
    g.close()


def test_stress_from_F_sweep_kernel():
    """Standalone sigma(F) over 2M random SPD-perturbed F, sampled against the
    oracle (sigma relative Frobenius <= 1e-4 per sample set)."""
    import torch
    from paper_2606_20426_gb300 import stress_from_F
    n = 2_000_000
    F = workloads.random_deformation_gradients(7, n)
    Ft = torch.from_numpy(F.reshape(n, 9).astype(np.float32)).cuda()
    sig = stress_from_F(Ft, 3e5, 0.45).cpu().numpy()
    mu, lam_hat, alpha = mat.snh_params(3e5, 0.45)
    idx = np.random.default_rng(0).choice(n, 4096, replace=False)
    F32 = F[idx].astype(np.float32).astype(np.float64)  # the GPU reads F in float32
    ref = mat.sym6(mat.cauchy(F32, mu, lam_hat, alpha))
    assert rel_fro(sig[:, idx].T, ref) <= 1e-4
    # ragged tail: the last elements are written too
    tail = np.arange(n - 5, n)
    ref_t = mat.sym6(mat.cauchy(F[tail].astype(np.float32).astype(np.float64), mu, lam_hat, alpha))
    assert rel_fro(sig[:, tail].T, ref_t) <= 1e-4


def test_stress_from_F_empty_and_tiny():
    import torch
    from paper_2606_20426_gb300 import stress_from_F
    out = stress_from_F(torch.zeros((0, 9), dtype=torch.float32, device="cuda"), 3e5, 0.45)
    assert out.shape == (6, 0)
    F = torch.eye(3, device="cuda").reshape(1, 9).repeat(3, 1).contiguous()
    assert float(stress_from_F(F, 3e5, 0.45).abs().max()) == 0.0


def test_no_grid_and_far_indenter():
    env = copy.deepcopy(workloads.small_env(0))
    env["grid"] = None
    env["start_pose"]["t"] = env["start_pose"]["t"] + np.array([0.0, 0.0, 0.01])
    for p in env["poses"]:
        p["t"] = p["t"] + np.array([0.0, 0.0, 0.01])
    g = _gpu_env(env)
    g.step(env["poses"][0])
    assert np.abs(g.contact_force()).max() == 0.0
    assert np.abs(g.positions() - env["X"]).max() == 0.0
    from paper_2606_20426_gb300 import TcError
    with pytest.raises(TcError):
        g.pressure_map()
    g.close()


def _other_grids(env):
    """Grids besides the create-time one: finer, coarser, shifted, and swapped
    axes (rows along the other side)."""
    g0 = env["grid"]
    out = []
    for (fh, fw), shift, swap in [((2, 2), (0.0, 0.0), False), ((0.5, 0.75), (0.0, 0.0), False),
                                  ((1, 1), (0.3, -0.2), False), ((1, 1), (0.0, 0.0), True),
                                  ((1.5, 1.25), (0.1, 0.1), False)]:
        H, W = max(1, int(g0["H"] * fh)), max(1, int(g0["W"] * fw))
        pix = (g0["pixel"][0] * g0["W"] / W, g0["pixel"][1] * g0["H"] / H)
        origin = (g0["origin"][0] + shift[0] * pix[0], g0["origin"][1] + shift[1] * pix[1])
        g = dict(axis_u=g0["axis_u"], axis_v=g0["axis_v"], origin=origin, pixel=pix, H=H, W=W)
        if swap:
            g = dict(axis_u=g0["axis_v"], axis_v=g0["axis_u"], origin=origin[::-1], pixel=pix[::-1], H=W, W=H)
        out.append(g)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pressure_map_on_caller_grids(precision):
    """tc_pressure_map(env, grid): each grid is binned on first use (masks
    bit-exact against the oracle's exact binning of that grid, maps within
    1e-3), kept (a second call is bit-identical), and more grids than the
    cache holds still give the right maps; NULL is the create-time grid;
    invalid grids are refused."""
    from paper_2606_20426_gb300 import TcError
    env = workloads.small_env(0, steps=1)
    g = _gpu_env(env, precision)
    g.step(env["poses"][0])
    x = g.positions()
    base, _ = g.pressure_map()
    grids = _other_grids(env)
    first = {}
    for rnd in range(2):
        for i, gr in enumerate(grids):
            e2 = dict(env)
            e2["grid"] = gr
            ref = Scene(e2)
            mref, mask_ref = ref.pressure_map(x=x)
            m, mask = g.pressure_map(grid=gr)
            m, mask = m.cpu().numpy(), mask.cpu().numpy()
            assert m.shape == (gr["H"], gr["W"])
            assert np.array_equal(mask, mask_ref)
            assert np.abs(mref).max() > 0 and rel_fro(m, mref) <= 1e-3
            if rnd == 0:
                first[i] = m
            else:
                assert np.array_equal(m, first[i])
    again, _ = g.pressure_map(grid=env["grid"])
    assert np.array_equal(again.cpu().numpy(), base.cpu().numpy())
    for bad in [dict(env["grid"], H=0), dict(env["grid"], axis_u=1, axis_v=1),
                dict(env["grid"], pixel=(0.0, 1e-3)), dict(env["grid"], axis_v=3)]:
        with pytest.raises(TcError) as ei:
            g.pressure_map(grid=bad, out=base.new_empty((max(bad["H"], 1), bad["W"])), mask=None, want_mask=False)
        assert ei.value.code == 1
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_extract_batch_equals_per_env_calls(precision):
    """tc_extract_batch over envs of different sizes (one cooperative launch)
    writes, bit for bit, what tc_stress and tc_pressure_map write per env,
    also when some envs ask for sigma only or the map only."""
    import torch
    from paper_2606_20426_gb300 import extract_batch
    cfgs = [workloads.small_env(0, steps=1), workloads.pad_env(2, steps=1), workloads.small_env(3, steps=1),
            workloads.gelsight_env(4, steps=1, target_tets=6000, grid_hw=(90, 120))]
    envs = [_gpu_env(c, precision) for c in cfgs]
    for g, c in zip(envs, cfgs):
        g.set_positions(_smooth_positions(c["X"], amp=5e-5, seed=len(c["X"])))
    ref = [(g.stress().clone(),) + tuple(t.clone() for t in g.pressure_map()) for g in envs]
    dev = "cuda"
    sig = [torch.full((6, g.info["nt"]), float("nan"), device=dev) for g in envs]
    maps = [torch.full((g.info["H"], g.info["W"]), float("nan"), device=dev) for g in envs]
    masks = [torch.full((g.info["H"], g.info["W"]), 9, dtype=torch.uint8, device=dev) for g in envs]
    extract_batch(envs, sig, maps, masks)
    for (s0, m0, k0), s1, m1, k1 in zip(ref, sig, maps, masks):
        assert torch.equal(s0, s1) and torch.equal(m0, m1) and torch.equal(k0, k1)
    # partial requests: sigma of envs 0 and 2 only, maps of 1 and 3 only
    sig2 = [torch.zeros_like(s) for s in sig]
    map2 = [torch.zeros_like(m) for m in maps]
    extract_batch(envs, [sig2[0], None, sig2[2], None], [None, map2[1], None, map2[3]], None)
    assert torch.equal(sig2[0], ref[0][0]) and torch.equal(sig2[2], ref[2][0])
    assert torch.equal(map2[1], ref[1][1]) and torch.equal(map2[3], ref[3][1])
    assert torch.count_nonzero(sig2[1]).item() == 0 and torch.count_nonzero(map2[0]).item() == 0
    # a batch of one
    one = torch.zeros_like(maps[3])
    extract_batch(envs[3:], None, [one], None)
    assert torch.equal(one, ref[3][1])
    # copies of the envs (same positions) thirteen to a batch: many env
    # changes inside every block's share of each kind of item, every other
    # env sigma only
    rep = envs + [_gpu_env(cfgs[i % 4], precision) for i in range(4, 13)]
    for i in range(4, 13):
        c = cfgs[i % 4]
        rep[i].set_positions(_smooth_positions(c["X"], amp=5e-5, seed=len(c["X"])))
    sig3 = [torch.full_like(sig[i % 4], float("nan")) for i in range(13)]
    map3 = [torch.full_like(maps[i % 4], float("nan")) if i % 2 == 0 else None for i in range(13)]
    extract_batch(rep, sig3, map3, None)
    for i in range(13):
        assert torch.equal(sig3[i], ref[i % 4][0])
        if map3[i] is not None:
            assert torch.equal(map3[i], ref[i % 4][1])
    for g in rep:
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_depth_map_bit_exact(precision):
    """tc_depth_map (the deformed surface's height field, Sec. III-D's depth)
    equals the oracle's z-buffer of the same deformed contact faces bit for
    bit (same FP64 operations in the same order, one rounding to FP32), at
    rest, after indentation steps, and on another grid."""
    cfgs = [workloads.small_env(1, steps=2), workloads.gelsight_env(3, steps=4, target_tets=4000, grid_hw=(60, 80))]
    for c in cfgs:
        g = _gpu_env(c, precision)
        ref = Scene(c)
        for k in range(3):
            if k:
                g.step(c["poses"][k - 1])
            x = g.positions()
            m, mask = g.depth_map()
            mref, mask_ref = ref.depth_map(x)
            assert np.array_equal(mask.cpu().numpy(), mask_ref)
            assert np.array_equal(m.cpu().numpy(), mref)
            if k == 2:
                gr = _other_grids(c)[3]
                m2, k2 = g.depth_map(grid=gr)
                r2, rk2 = ref.depth_map(x, grid=gr)
                assert np.array_equal(k2.cpu().numpy(), rk2) and np.array_equal(m2.cpu().numpy(), r2)
        # pressed: the surface under the indenter is below the rest height
        assert mref[mask_ref == 1].min() < ref.X[:, 2].max() - 0.5 * c["depth"] / 2
        g.close()
