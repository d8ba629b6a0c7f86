"""Pins for oracle/sim.py: element gradient/Hessian against finite
differences, the linear patch test, energy decrease, no interpenetration,
quasi-static equilibrium (contact force = -support reaction), the sparse solve
against a dense one, the dynamic step and the traction identities of Eq. 5-8."""
import copy

import numpy as np
import pytest

from oracle import material as mat
from oracle import mesh as msh
from oracle.sim import Scene, InitialPenetration
from synth import workloads


@pytest.fixture(scope="module")
def stepped():
    env = workloads.small_env(1)
    sc = Scene(env)
    dmins = []
    for pose in env["poses"]:
        sc.step(pose)
        dmins.append(sc.min_distance(sc.x, sc.indenter(sc.pose)))
    return env, sc, dmins


def test_elastic_gradient_and_hessian_fd():
    env = workloads.small_env(0)
    sc = Scene(env)
    rng = np.random.default_rng(0)
    x = sc.X + 2e-5 * rng.standard_normal(sc.X.shape)
    _, ge, _ = sc.elastic(x)
    g = np.zeros((sc.nv, 3))
    np.add.at(g, sc.T.ravel(), ge.reshape(-1, 3))
    h = 1e-9
    for v, k in [(3, 0), (17, 2), (40, 1), (60, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[v, k] += h
        xm[v, k] -= h
        fd = (sc.elastic(xp, False)[0] - sc.elastic(xm, False)[0]) / (2 * h)
        assert fd == pytest.approx(g[v, k], rel=1e-5, abs=1e-9)
    # unprojected element Hessian = FD of the element gradient
    F = msh.deformation_gradient(x, sc.T, sc.Dminv)
    T9 = mat.dpk1_dF(F, sc.mu, sc.lam_hat, sc.alpha)
    He = sc.vol[:, None, None] * np.einsum("nki,nkl,nlj->nij", sc.Dfx, T9, sc.Dfx)
    e = 5
    for j in (0, 4, 11):
        d = np.zeros(12)
        d[j] = 1e-9
        def grad_e(dx):
            xx = x.copy()
            xx[sc.T[e]] += dx.reshape(4, 3)
            Fe = msh.deformation_gradient(xx, sc.T[e:e + 1], sc.Dminv[e:e + 1])
            P = mat.pk1(Fe, sc.mu, sc.lam_hat, sc.alpha).reshape(-1, 9)
            return sc.vol[e] * sc.Dfx[e].T @ P[0]
        fd = (grad_e(d) - grad_e(-d)) / 2e-9
        assert np.allclose(fd, He[e][:, j], rtol=1e-5, atol=1e-3)
    # the projected element Hessians are PSD
    _, _, Hp = sc.elastic(x)
    assert np.linalg.eigvalsh(Hp).min() > -1e-8 * np.abs(Hp).max()


def test_linear_patch_test():
    """Every boundary vertex prescribed to x = A X + c: the interior converges
    to the affine map and sigma is uniform and equal to sigma(A)."""
    env = copy.deepcopy(workloads.small_env(0, nx=3, ny=3, nz=3, size=(6e-3, 6e-3, 6e-3)))
    faces, _ = msh.boundary_faces(env["tets"])
    env["fixed"] = np.unique(faces.ravel()).astype(np.int32)
    env["start_pose"]["t"] = env["start_pose"]["t"] + np.array([0, 0, 0.05])  # far away
    sc = Scene(env)
    A = np.array([[1.02, 0.01, -0.005], [0.003, 0.985, 0.01], [0.0, -0.01, 1.03]])
    c = np.array([1e-4, -2e-4, 3e-4])
    x = sc.X.copy()
    x[sc.fixed] = sc.X[sc.fixed] @ A.T + c
    xs, _ = sc.newton(x, sc.indenter(sc.pose))
    target = sc.X @ A.T + c
    assert np.abs(xs - target).max() < 1e-10  # Newton tolerance, 6 mm cube
    sig = sc.stress(xs)
    ref = mat.sym6(mat.cauchy(A[None], sc.mu, sc.lam_hat, sc.alpha))[0]
    assert np.abs(sig - ref).max() < 1e-6 * np.abs(ref).max()
    assert all(np.all(np.diff(t) <= 0) for t in sc.trace)


def test_step_energy_monotone_and_separated(stepped):
    env, sc, dmins = stepped
    assert all(np.all(np.diff(t) <= 0) for t in sc.trace if len(t) > 1)
    assert min(dmins) > 0.0
    assert sc.separated(sc.x, sc.indenter(sc.pose))
    # the pad was pressed: contact force points into the gel (-z)
    assert sc.contact_force()[2] < -1e-3


def test_quasistatic_equilibrium(stepped):
    """Newton converged to a stationary point: the force the indenter applies
    is carried by the fixed support."""
    _, sc, _ = stepped
    f = sc.contact_force()
    r = sc.reaction_force()
    assert np.abs(f + r).max() < 1e-5 * np.abs(f).max()


def test_sparse_solve_matches_dense(stepped):
    import scipy.sparse.linalg as spla
    _, sc, _ = stepped
    E, g, H = sc.gradient_hessian(sc.x, sc.indenter(sc.pose))
    fr = np.repeat(sc.free, 3)
    Hff = H[fr][:, fr]
    rhs = np.random.default_rng(0).standard_normal(Hff.shape[0])
    xs = spla.spsolve(Hff.tocsc(), rhs)
    xd = np.linalg.solve(Hff.toarray(), rhs)
    assert np.allclose(xs, xd, rtol=1e-8, atol=1e-12 * np.abs(xd).max())
    w = np.linalg.eigvalsh(Hff.toarray())
    assert w.min() > 0  # projected Hessian + fixed set: SPD


def test_traction_identities(stepped):
    _, sc, _ = stepped
    t, p, tt = sc.traction()
    f = sc.cfaces
    c = np.cross(sc.x[f[:, 1]] - sc.x[f[:, 0]], sc.x[f[:, 2]] - sc.x[f[:, 0]])
    n = c / np.linalg.norm(c, axis=1, keepdims=True)
    assert np.abs(np.einsum("ij,ij->i", tt, n)).max() < 1e-9 * np.abs(t).max()   # Eq. 8
    assert np.allclose(t, tt - p[:, None] * n, atol=1e-9 * np.abs(t).max())
    # top faces point up (outward) in the rest state
    c0 = np.cross(sc.X[f[:, 1]] - sc.X[f[:, 0]], sc.X[f[:, 2]] - sc.X[f[:, 0]])
    assert np.all(c0[:, 2] > 0)
    # compression under the indenter: positive pressure somewhere
    assert p.max() > 0
    m, mask = sc.pressure_map()
    assert mask.sum() == m.size and np.isfinite(m).all()


def test_affine_field_pressure_is_uniform():
    """Under a homogeneous deformation every top face carries
    p = -n.sigma(A) n and every pixel shows the same value."""
    env = workloads.small_env(0)
    sc = Scene(env)
    A = np.array([[1.01, 0.0, 0.0], [0.0, 0.99, 0.0], [0.002, 0.0, 0.97]])
    x = sc.X @ A.T
    S = mat.cauchy(A[None], sc.mu, sc.lam_hat, sc.alpha)[0]
    n = np.linalg.inv(A).T @ np.array([0, 0, 1.0])
    n /= np.linalg.norm(n)
    _, p, _ = sc.traction(x)
    assert np.allclose(p, -n @ S @ n, rtol=1e-10)
    m, _ = sc.pressure_map(x)
    assert np.allclose(m, -n @ S @ n, rtol=1e-6)


def test_dynamic_step_runs_and_balances_momentum():
    env = workloads.small_env(2, dt=1.0 / 60.0, steps=1)
    sc = Scene(env)
    sc.step(env["poses"][0])
    assert all(np.all(np.diff(t) <= 0) for t in sc.trace if len(t) > 1)
    assert np.isfinite(sc.v).all() and np.abs(sc.v[sc.fixed]).max() == 0.0


def test_initial_penetration_rejected():
    env = copy.deepcopy(workloads.small_env(0))
    env["start_pose"]["t"] = env["start_pose"]["t"] - np.array([0, 0, 0.5e-3])
    with pytest.raises(InitialPenetration):
        Scene(env)
