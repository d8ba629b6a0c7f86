"""Pins for the full stable Neo-Hookean law of oracle/material.py (Smith et
al. 2018, the law Sec. III-B cites, with its log term): the rest state is
stress-free, the small-strain limit is linear elasticity with Eq. 1's
(E, nu) (which fixes both the 4/3, 5/6 parameter map and the log term's
coefficient), P and the tangent against central differences of the energy,
Eq. 3 against the closed-form Cauchy stress, symmetry and objectivity, the
energy's finiteness at a collapsed element, and whole-scene checks (the
linear patch test and the FD gradient of the scene's elastic energy)."""
import copy

import numpy as np
import pytest

from oracle import material as mat
from oracle import mesh as msh
from oracle.sim import Scene
from synth import workloads

E, NU = 3.0e5, 0.45
MP = mat.snh_log_params(E, NU)


def rand_F(rng, n, scale=0.3):
    return np.eye(3) + scale * rng.standard_normal((n, 3, 3))


@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45, 0.49])
def test_rest_state_is_stress_free(nu):
    mp = mat.snh_log_params(E, nu)
    I = np.eye(3)[None]
    assert abs(mat.energy_density_log(I, *mp)[0]) < 1e-9 * E
    assert np.abs(mat.pk1_log(I, *mp)).max() < 1e-9 * E
    assert np.abs(mat.cauchy_log(I, *mp)).max() < 1e-9 * E


@pytest.mark.parametrize("nu", [0.2, 0.45])
def test_small_strain_limit_matches_linear_elasticity(nu):
    """sigma(I + eps H) / eps -> 2 mu sym(H) + lam tr(H) I with Eq. 1's
    (mu, lam); a log term with another coefficient or argument, or another
    parameter map, gives other limits."""
    rng = np.random.default_rng(12)
    mu, lam = mat.lame(E, nu)
    mp = mat.snh_log_params(E, nu)
    for _ in range(3):
        H = rng.standard_normal((3, 3))
        eps = 1e-6
        sig = mat.cauchy_log((np.eye(3) + eps * H)[None], *mp)[0] / eps
        lin = mu * (H + H.T) + lam * np.trace(H) * np.eye(3)
        assert np.abs(sig - lin).max() < 1e-4 * np.abs(lin).max()


def test_pk1_is_energy_gradient():
    rng = np.random.default_rng(13)
    F = rand_F(rng, 8)
    h = 1e-6
    P = mat.pk1_log(F, *MP)
    for i in range(3):
        for j in range(3):
            d = np.zeros((3, 3))
            d[i, j] = h
            fd = (mat.energy_density_log(F + d, *MP) - mat.energy_density_log(F - d, *MP)) / (2 * h)
            assert np.allclose(fd, P[:, i, j], rtol=1e-6, atol=1e-4)


def test_tangent_is_pk1_derivative():
    rng = np.random.default_rng(14)
    F = rand_F(rng, 8)
    h = 1e-6
    T = mat.dpk1_dF_log(F, *MP)
    for k in range(9):
        d = np.zeros(9)
        d[k] = h
        d = d.reshape(3, 3)
        fd = (mat.pk1_log(F + d, *MP) - mat.pk1_log(F - d, *MP)).reshape(-1, 9) / (2 * h)
        assert np.allclose(fd, T[:, :, k], rtol=1e-6, atol=1e-3)
    assert np.abs(T - np.swapaxes(T, 1, 2)).max() < 1e-6


def test_eq3_equals_closed_form_cauchy():
    rng = np.random.default_rng(15)
    F = rand_F(rng, 16)
    F = F[np.linalg.det(F) > 0.2]
    ref = mat.cauchy_from_pk1(F, mat.pk1_log(F, *MP))
    assert np.allclose(mat.cauchy_log(F, *MP), ref, rtol=1e-10, atol=1e-9 * E)


def test_symmetry_and_objectivity():
    rng = np.random.default_rng(16)
    F = rand_F(rng, 6)
    F = F[np.linalg.det(F) > 0.2]
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    q *= np.sign(np.linalg.det(q))
    s = mat.cauchy_log(F, *MP)
    sr = mat.cauchy_log(q @ F, *MP)
    assert np.abs(s - np.swapaxes(s, 1, 2)).max() < 1e-9
    assert np.abs(sr - q @ s @ q.T).max() < 1e-8 * np.abs(s).max()
    # the energy is isotropic too: Psi(F Q) = Psi(F)
    assert np.allclose(mat.energy_density_log(F @ q, *MP), mat.energy_density_log(F, *MP), rtol=1e-10)


def test_log_term_keeps_collapse_finite_and_differs_from_the_rest_stable_law():
    """With the +1 inside the log, Psi stays finite at F = 0 (and P(0) = 0);
    the law agrees with the rest-stable law only to first order."""
    Z = np.zeros((1, 3, 3))
    assert np.isfinite(mat.energy_density_log(Z, *MP)[0])
    assert np.abs(mat.pk1_log(Z, *MP)).max() == 0.0
    mu, lam_hat, alpha = mat.law_params("snh", E, NU)
    F = np.diag([1.3, 0.9, 0.95])[None]
    a, b = mat.cauchy_log(F, *MP)[0], mat.cauchy(F, mu, lam_hat, alpha)[0]
    assert np.abs(a - b).max() > 1e-3 * np.abs(b).max()


def _log_env(**kw):
    env = copy.deepcopy(workloads.small_env(0, **kw))
    env["material"] = dict(env["material"], model="snh_log")
    return env


def test_scene_gradient_and_patch_test():
    """The scene's elastic gradient is the FD of its energy under the log
    law, and the linear patch test holds with sigma = sigma_log(A)."""
    sc = Scene(_log_env())
    assert sc.law == "snh_log"
    rng = np.random.default_rng(17)
    x = sc.X + 2e-5 * rng.standard_normal(sc.X.shape)
    _, ge, Hp = sc.elastic(x)
    g = np.zeros((sc.nv, 3))
    np.add.at(g, sc.T.ravel(), ge.reshape(-1, 3))
    h = 1e-9
    for v, k in [(3, 0), (17, 2), (40, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[v, k] += h
        xm[v, k] -= h
        fd = (sc.elastic(xp, False)[0] - sc.elastic(xm, False)[0]) / (2 * h)
        assert fd == pytest.approx(g[v, k], rel=1e-5, abs=1e-9)
    assert np.linalg.eigvalsh(Hp).min() > -1e-8 * np.abs(Hp).max()

    env = _log_env(nx=3, ny=3, nz=3, size=(6e-3, 6e-3, 6e-3))
    faces, _ = msh.boundary_faces(env["tets"])
    env["fixed"] = np.unique(faces.ravel()).astype(np.int32)
    env["start_pose"]["t"] = env["start_pose"]["t"] + np.array([0, 0, 0.05])
    sc = Scene(env)
    A = np.array([[1.02, 0.01, -0.005], [0.003, 0.985, 0.01], [0.0, -0.01, 1.03]])
    c = np.array([1e-4, -2e-4, 3e-4])
    x = sc.X.copy()
    x[sc.fixed] = sc.X[sc.fixed] @ A.T + c
    xs, _ = sc.newton(x, sc.indenter(sc.pose))
    assert np.abs(xs - (sc.X @ A.T + c)).max() < 1e-10
    ref = mat.sym6(mat.cauchy_log(A[None], *MP))[0]
    assert np.abs(sc.stress(xs) - ref).max() < 1e-6 * np.abs(ref).max()


def test_unknown_law_is_rejected():
    env = copy.deepcopy(workloads.small_env(0))
    env["material"] = dict(env["material"], model="mooney")
    with pytest.raises(ValueError):
        Scene(env)
