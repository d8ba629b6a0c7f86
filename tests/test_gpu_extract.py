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
