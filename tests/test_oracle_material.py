"""Pins for oracle/material.py: Eq. 1 against a hand-evaluated fixture,
Eq. 3 against Eq. 4, closed-form stresses for homogeneous deformations,
symmetry, objectivity, the small-strain limit, and finite differences."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import material as mat

E, NU = 3.0e5, 0.45
MU, LAM_HAT, ALPHA = mat.snh_params(E, NU)
GOLD = os.path.join(os.path.dirname(__file__), "golden", "lame_E0.3MPa_nu0.45.txt")


def _gold():
    vals = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = v
    return {k: Fraction(int(vals[k + "_num"]), int(vals[k + "_den"]))
            for k in ("mu", "lam", "lam_hat", "alpha")}


def rand_F(rng, n, scale=0.3):
    return np.eye(3) + scale * rng.standard_normal((n, 3, 3))


def test_lame_fixture():
    g = _gold()
    mu, lam = mat.lame(E, NU)
    assert mu == pytest.approx(float(g["mu"]), rel=1e-15)
    assert lam == pytest.approx(float(g["lam"]), rel=1e-15)
    assert LAM_HAT == pytest.approx(float(g["lam_hat"]), rel=1e-15)
    assert ALPHA == pytest.approx(float(g["alpha"]), rel=1e-15)


def test_rest_state_is_stress_free():
    I = np.eye(3)[None]
    assert abs(mat.energy_density(I, MU, LAM_HAT, ALPHA)[0]) < 1e-9
    assert np.abs(mat.pk1(I, MU, LAM_HAT, ALPHA)).max() < 1e-9
    assert np.abs(mat.cauchy(I, MU, LAM_HAT, ALPHA)).max() < 1e-9
    # the printed Eq. 4 is not stress-free at rest (the reason for the reading)
    mu, lam = mat.lame(E, NU)
    assert np.allclose(mat.sigma_paper_literal(I, mu, lam)[0], mu * np.eye(3))


def test_eq3_equals_eq4():
    rng = np.random.default_rng(0)
    F = rand_F(rng, 200)
    F = F[np.linalg.det(F) > 0.2]
    s3 = mat.cauchy_from_pk1(F, mat.pk1(F, MU, LAM_HAT, ALPHA))
    s4 = mat.cauchy(F, MU, LAM_HAT, ALPHA)
    assert np.abs(s3 - s4).max() < 1e-9 * np.abs(s4).max()


@pytest.mark.parametrize("s", [0.8, 0.95, 1.0, 1.07, 1.3])
def test_hydrostatic(s):
    sig = mat.cauchy(s * np.eye(3)[None], MU, LAM_HAT, ALPHA)[0]
    assert np.allclose(sig, (MU / s + LAM_HAT * (s ** 3 - ALPHA)) * np.eye(3), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("s", [0.85, 1.1, 1.25])
def test_uniaxial_strain(s):
    sig = mat.cauchy(np.diag([s, 1.0, 1.0])[None], MU, LAM_HAT, ALPHA)[0]
    assert sig[0, 0] == pytest.approx(MU * s + LAM_HAT * (s - ALPHA), rel=1e-12)
    assert sig[1, 1] == pytest.approx(MU / s + LAM_HAT * (s - ALPHA), rel=1e-12)
    assert sig[2, 2] == pytest.approx(MU / s + LAM_HAT * (s - ALPHA), rel=1e-12)
    assert np.abs(sig - np.diag(np.diag(sig))).max() < 1e-9


@pytest.mark.parametrize("s", [0.9, 1.05, 1.2])
def test_uniaxial_stress(s):
    J = ALPHA - MU / (LAM_HAT * s)
    t = np.sqrt(J / s)
    sig = mat.cauchy(np.diag([s, t, t])[None], MU, LAM_HAT, ALPHA)[0]
    assert abs(sig[1, 1]) < 1e-9 * MU and abs(sig[2, 2]) < 1e-9 * MU
    assert sig[0, 0] == pytest.approx(MU * (s * s - t * t) / J, rel=1e-12)


@pytest.mark.parametrize("gamma", [0.01, 0.2, 0.5])
def test_simple_shear(gamma):
    F = np.eye(3)
    F[0, 1] = gamma
    sig = mat.cauchy(F[None], MU, LAM_HAT, ALPHA)[0]
    assert sig[0, 1] == pytest.approx(MU * gamma, rel=1e-12)
    assert sig[0, 0] == pytest.approx(MU * gamma ** 2, rel=1e-10)
    assert abs(sig[1, 1]) < 1e-6 and abs(sig[2, 2]) < 1e-6


def test_symmetry_and_objectivity():
    rng = np.random.default_rng(1)
    F = rand_F(rng, 50, 0.2)
    q, _ = np.linalg.qr(rng.standard_normal((50, 3, 3)))
    q = q * np.sign(np.linalg.det(q))[:, None, None]
    s = mat.cauchy(F, MU, LAM_HAT, ALPHA)
    sr = mat.cauchy(q @ F, MU, LAM_HAT, ALPHA)
    assert np.abs(s - np.swapaxes(s, 1, 2)).max() < 1e-9
    assert np.abs(sr - q @ s @ np.swapaxes(q, 1, 2)).max() < 1e-8 * np.abs(s).max()


def test_small_strain_limit_matches_linear_elasticity():
    """sigma(I + eps H) / eps -> 2 mu sym(H) + lam tr(H) I with Eq. 1's (mu, lam)."""
    rng = np.random.default_rng(2)
    mu, lam = mat.lame(E, NU)
    H = rng.standard_normal((3, 3))
    eps = 1e-6
    sig = mat.cauchy((np.eye(3) + eps * H)[None], MU, LAM_HAT, ALPHA)[0] / eps
    lin = mu * (H + H.T) + lam * np.trace(H) * np.eye(3)
    assert np.abs(sig - lin).max() < 1e-4 * np.abs(lin).max()


def test_pk1_is_energy_gradient():
    rng = np.random.default_rng(3)
    F = rand_F(rng, 8)
    h = 1e-6
    P = mat.pk1(F, MU, LAM_HAT, ALPHA)
    for i in range(3):
        for j in range(3):
            d = np.zeros((3, 3))
            d[i, j] = h
            fd = (mat.energy_density(F + d, MU, LAM_HAT, ALPHA) - mat.energy_density(F - d, MU, LAM_HAT, ALPHA)) / (2 * h)
            assert np.allclose(fd, P[:, i, j], rtol=1e-6, atol=1e-4)


def test_tangent_is_pk1_derivative():
    rng = np.random.default_rng(4)
    F = rand_F(rng, 8)
    h = 1e-6
    T = mat.dpk1_dF(F, MU, LAM_HAT, ALPHA)
    for k in range(9):
        d = np.zeros(9)
        d[k] = h
        d = d.reshape(3, 3)
        fd = (mat.pk1(F + d, MU, LAM_HAT, ALPHA) - mat.pk1(F - d, MU, LAM_HAT, ALPHA)).reshape(-1, 9) / (2 * h)
        assert np.allclose(fd, T[:, :, k], rtol=1e-6, atol=1e-3)
    assert np.abs(T - np.swapaxes(T, 1, 2)).max() < 1e-6


def test_cofactor_matches_inverse_transpose():
    rng = np.random.default_rng(5)
    F = rand_F(rng, 20)
    F = F[np.abs(np.linalg.det(F)) > 0.1]
    ref = np.linalg.det(F)[:, None, None] * np.swapaxes(np.linalg.inv(F), 1, 2)
    assert np.allclose(mat.cofactor(F), ref, atol=1e-12)


def test_project_psd():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((10, 9, 9))
    A = A + np.swapaxes(A, 1, 2)
    P = mat.project_psd(A)
    w = np.linalg.eigvalsh(P)
    assert w.min() > -1e-10 * np.abs(A).max()
    S = A @ np.swapaxes(A, 1, 2)  # already PSD: projection is the identity
    assert np.allclose(mat.project_psd(S), S, atol=1e-10)
    # the rest-state tangent has a zero (rotation) mode and nothing negative
    T0 = mat.dpk1_dF(np.eye(3)[None], MU, LAM_HAT, ALPHA)[0]
    w0 = np.linalg.eigvalsh(T0)
    assert w0.min() > -1e-6 * MU and abs(w0[:3]).max() < 1e-6 * MU


def test_sym6_roundtrip():
    rng = np.random.default_rng(7)
    S = rng.standard_normal((4, 3, 3))
    S = S + np.swapaxes(S, 1, 2)
    assert np.allclose(mat.full33(mat.sym6(S)), S)


# ------------------------------------------------- heterogeneous material

def test_per_tet_material_equals_homogeneous_when_uniform():
    """A per-tet (E, nu) table with every entry equal to the scene's material
    gives the homogeneous scene's energy, gradient and stress."""
    import copy
    from oracle.sim import Scene
    from synth import workloads
    env = workloads.small_env(0)
    het = copy.deepcopy(env)
    het["material"]["per_tet"] = np.tile([env["material"]["E"], env["material"]["nu"]], (len(env["tets"]), 1))
    a, b = Scene(env), Scene(het)
    x = a.X + 1e-5 * np.sin(500 * a.X[:, [1, 2, 0]])
    Ea, ga, Ha = a.elastic(x)
    Eb, gb, Hb = b.elastic(x)
    assert Eb == pytest.approx(Ea, rel=1e-14)
    assert np.allclose(gb, ga, rtol=1e-13, atol=1e-25) and np.allclose(Hb, Ha, rtol=1e-12, atol=1e-20)
    assert np.allclose(b.stress(x), a.stress(x), rtol=1e-13, atol=1e-12)


def test_two_layers_each_follow_their_own_closed_form():
    """Under a homogeneous uniaxial strain F = diag(1, 1, s) every tet of a
    dual-layer pad shows the closed-form sigma_zz = mu s + lam_hat (s - alpha)
    and sigma_xx = mu / s + lam_hat (s - alpha) of its own layer's (E, nu),
    and the element gradients match central differences of the energy."""
    from oracle.sim import Scene
    from synth import workloads
    env = workloads.small_env(0)
    env["material"]["per_tet"] = workloads.dual_layer_material(env["X"], env["tets"], top_thickness=1e-3,
                                                               E_top=0.2e6, E_base=0.9e6, nu=0.4)
    sc = Scene(env)
    s = 0.97
    x = sc.X * np.array([1.0, 1.0, s])
    sig = sc.stress(x)
    pt = env["material"]["per_tet"]
    for E in (0.2e6, 0.9e6):
        mu, lh, al = mat.snh_params(E, 0.4)
        sel = pt[:, 0] == E
        assert sel.sum() > 10
        assert np.allclose(sig[sel, 2], mu * s + lh * (s - al), rtol=1e-12)
        assert np.allclose(sig[sel, 0], mu / s + lh * (s - al), rtol=1e-12)
    rng = np.random.default_rng(1)
    x = sc.X + 2e-5 * rng.standard_normal(sc.X.shape)
    _, ge, _ = sc.elastic(x)
    g = np.zeros((sc.nv, 3))
    np.add.at(g, sc.T.ravel(), ge.reshape(-1, 3))
    h = 1e-9
    for v, k in [(5, 2), (30, 0), (61, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[v, k] += h
        xm[v, k] -= h
        assert (sc.elastic(xp, False)[0] - sc.elastic(xm, False)[0]) / (2 * h) == pytest.approx(g[v, k], rel=1e-5)
