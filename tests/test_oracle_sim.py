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


# ------------------------------------------------------------------ inertia
# The dynamic branch of the incremental potential (Algorithm 2's step at
# dt > 0): E(x) = 1/(2 h^2) |x - x_tilde|_M^2 + elastic + barrier with
# x_tilde = x_t + h v_t, and the update v = (x - x_t) / h.  Mechanics fixes
# what implicit Euler must give without contact: a rigid translation is
# exact, total momentum is conserved when nothing is fixed, and a linear
# oscillator follows (I + h^2 M^-1 K)^-1 (x_t + h v_t).

def _free_floating(seed=3, dt=1.0 / 60.0):
    """small_env with nothing fixed and the indenter 10 mm above the pad (no
    contact pair can form), for the inertia pins."""
    env = copy.deepcopy(workloads.small_env(seed, dt=dt, steps=1))
    env["fixed"] = np.zeros(0, dtype=np.int32)
    env["start_pose"]["t"] = env["start_pose"]["t"] + np.array([0.0, 0.0, 10e-3])
    env["poses"] = [copy.deepcopy(env["start_pose"]) for _ in range(3)]
    env["grid"] = None
    return env


def _lumped_mass(X, T, rho):
    """rho V / 4 to each corner, V = det[X1-X0, X2-X0, X3-X0] / 6 (textbook
    lumped mass, computed here without the oracle's mesh module)."""
    m = np.zeros(len(X))
    for t in T:
        V = np.linalg.det(np.stack([X[t[1]] - X[t[0]], X[t[2]] - X[t[0]], X[t[3]] - X[t[0]]], axis=1)) / 6.0
        m[t] += rho * V / 4.0
    return m


def test_inertia_rigid_translation_is_exact():
    """Uniform v0 and no constraint: every step moves the body by h v0 and
    keeps v = v0 (the elastic energy of a translation is zero, so x_tilde
    itself is the minimiser)."""
    env = _free_floating()
    sc = Scene(env)
    h = env["opts"]["dt"]
    v0 = np.array([3e-3, -2e-3, 1e-3])
    sc.v = np.tile(v0, (sc.nv, 1))
    for k in range(1, 4):
        sc.step(env["poses"][k - 1])
        assert np.abs(sc.x - (sc.X + k * h * v0)).max() <= 1e-12
        assert np.abs(sc.v - v0).max() <= 1e-9 * np.abs(v0).max()


def test_inertia_conserves_total_momentum():
    """No fixed vertex and no contact: internal forces sum to zero, so
    implicit Euler keeps sum_v m_v v_v (lumped masses) exactly; a wrong mass
    vector or an x_tilde without h v_t breaks it."""
    env = _free_floating(seed=5)
    sc = Scene(env)
    rng = np.random.default_rng(11)
    v0 = 2e-3 * rng.standard_normal((sc.nv, 3))       # stretching + shearing field
    sc.v = v0.copy()
    m = _lumped_mass(sc.X, sc.T, env["material"]["density"])
    p0 = (m[:, None] * v0).sum(axis=0)
    sc.step(env["poses"][0])
    p1 = (m[:, None] * sc.v).sum(axis=0)
    assert np.abs(sc.x - sc.X).max() > 1e-6             # the body deformed
    assert np.abs(p1 - p0).max() <= 1e-8 * np.abs(m[:, None] * v0).sum(axis=0).max()
    # the velocity field changed (elastic forces acted), momentum did not
    assert np.abs(sc.v - v0).max() > 1e-2 * np.abs(v0).max()


def test_implicit_euler_one_free_vertex_closed_form():
    """One tet, three base vertices fixed, the apex free.  For small motion the
    apex is a 3-D linear oscillator with stiffness K = V [mu |n|^2 I +
    (lam + mu) n n^T] (linear elasticity with Eq. 1's Lame parameters, the
    small-strain limit of the material) and lumped mass m = rho V / 4; implicit
    Euler gives u_{k+1} = (I + h^2 K / m)^-1 (u_k + h v_k).  h is chosen so that
    h^2 K / m is of order one, so a wrong power of h fails."""
    L = 1e-3
    X = np.array([[0.0, 0.0, 0.0], [L, 0.0, 0.0], [0.0, L, 0.0], [0.3 * L, 0.35 * L, L]])
    T = np.array([[0, 1, 2, 3]], dtype=np.int32)
    E, nu, rho = 3.0e5, 0.45, 1100.0
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    V = L ** 3 / 6.0
    # gradient of the apex's barycentric (hat) function: N(X_a) = 1, 0 elsewhere
    c = np.linalg.solve(np.hstack([X, np.ones((4, 1))]), np.array([0.0, 0.0, 0.0, 1.0]))
    n = c[:3]
    K = V * (mu * (n @ n) * np.eye(3) + (lam + mu) * np.outer(n, n))
    m = rho * V / 4.0
    h = float(np.sqrt(m / np.linalg.eigvalsh(K).mean()))
    Vi, Fi = workloads.indenters.icosphere(1e-3, 1)
    pose = dict(R=np.eye(3), t=np.array([0.3 * L, 0.35 * L, 20e-3]))
    env = dict(X=X, tets=T, material=dict(E=E, nu=nu, density=rho), fixed=np.array([0, 1, 2], dtype=np.int32),
               ind_V=Vi, ind_F=Fi, start_pose=pose, grid=None,
               opts=dict(dhat=0.05e-3, kappa=1.0, dt=h, newton_rtol=1e-10, newton_max=50))
    sc = Scene(env)
    v0 = np.array([2e-4, -1e-4, 3e-4])                 # h v0 ~ 1e-8 m: strain ~1e-5
    sc.v[3] = v0
    A = np.linalg.inv(np.eye(3) + h * h * K / m)
    u, v = np.zeros(3), v0.copy()
    for _ in range(2):
        u_next = A @ (u + h * v)
        sc.step(pose)
        got = sc.x[3] - X[3]
        assert np.linalg.norm(got - u_next) <= 1e-4 * np.linalg.norm(u_next)
        assert np.linalg.norm(sc.v[3] - (u_next - u) / h) <= 1e-4 * np.linalg.norm(v0)
        u, v = u_next, (u_next - u) / h
    assert np.abs(sc.x[:3] - X[:3]).max() == 0.0


# -------------------------------------------------- area weighting and map
# R7 reading (vertex value = sum_f A_f p_f / sum_f A_f over the incident
# contact faces, deformed areas) and the pixel gather of the pressure map.

def _bare_scene(X, faces):
    sc = Scene.__new__(Scene)
    sc.X = np.asarray(X, dtype=np.float64)
    sc.x = sc.X.copy()
    sc.cfaces = np.asarray(faces, dtype=np.int64)
    sc.cverts, sc.csr_off, sc.csr_idx = msh.vertex_face_csr(sc.cfaces)
    return sc


def test_vertex_pressure_worked_example_deformed_areas():
    """A three-face fan with deformed areas 1/2, 1 and 3 (mm^2) carrying
    p = 1, 2, 5: the hub's value is (1/2 + 2 + 15) / (9/2) = 35/9 (an
    unweighted mean gives 8/3, rest areas -- all equal here -- give 8/3)."""
    mm = 1e-3
    x = mm * np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-2, 0, 0], [0, -3, 0]], dtype=np.float64)
    X = mm * np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]], dtype=np.float64)
    faces = [[0, 1, 2], [0, 2, 3], [0, 3, 4]]
    sc = _bare_scene(X, faces)
    pv = sc.vertex_pressure(x=x, p_face=np.array([1.0, 2.0, 5.0]))
    # slots follow sorted vertex ids 0..4
    expect = np.array([35 / 9, 1.0, 5 / 3, 17 / 4, 5.0])
    assert np.allclose(pv, expect, rtol=1e-14)


def test_vertex_pressure_invariant_under_face_split():
    """Splitting a face of the hub's fan into two faces with the same pressure
    leaves the hub's weighted mean unchanged (a face counts by its area, not
    by its count); vertices 1 and 2, whose fans are untouched, keep theirs."""
    mm = 1e-3
    x = mm * np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-2, 0, 0], [0, -3, 0], [-1, -1.5, 0]], dtype=np.float64)
    whole = _bare_scene(x[:5], [[0, 1, 2], [0, 2, 3], [0, 3, 4]])
    split = _bare_scene(x, [[0, 1, 2], [0, 2, 3], [0, 3, 5], [0, 5, 4]])
    a = whole.vertex_pressure(x=x[:5], p_face=np.array([1.0, 2.0, 5.0]))
    b = split.vertex_pressure(x=x, p_face=np.array([1.0, 2.0, 5.0, 5.0]))
    assert np.allclose(b[:3], a[:3], rtol=1e-14)
    assert b[0] == pytest.approx(35 / 9, rel=1e-14)
    # vertex 3 now sees only the half (area 3/2) of the split face: (2 + 7.5) / 2.5
    assert b[3] == pytest.approx(3.8, rel=1e-14)


def _pixel_centres(grid):
    H, W = grid["H"], grid["W"]
    u = grid["origin"][0] + (np.arange(W) + 0.5) * grid["pixel"][0]
    v = grid["origin"][1] + (np.arange(H) + 0.5) * grid["pixel"][1]
    return np.meshgrid(u, v)  # (H, W) each: u along columns, v along rows


@pytest.mark.parametrize("which", ["pad", "graded"])
def test_pressure_map_reproduces_linear_vertex_field(which):
    """Barycentric interpolation reproduces a linear field exactly: with
    p_v = a . (u_v, v_v) + b at the contact vertices (rest coordinates in the
    grid plane), every covered pixel shows a . (u_c, v_c) + b at its centre.
    A permuted vertex slot, a wrong weight order or swapped grid axes fails."""
    if which == "pad":
        env = workloads.pad_env(0, steps=1)
    else:
        env = workloads.gelsight_env(2, steps=1, target_tets=4000, grid_hw=(30, 40))
    sc = Scene(env)
    g = env["grid"]
    a, b = np.array([2.0e5, -7.0e5]), 30.0
    Xc = sc.X[sc.cverts]
    pv = a[0] * Xc[:, g["axis_u"]] + a[1] * Xc[:, g["axis_v"]] + b
    m, mask = sc.pressure_map(p_vertex=pv)
    U, Vv = _pixel_centres(g)
    expect = a[0] * U + a[1] * Vv + b
    cov = mask.astype(bool)
    assert cov.mean() > 0.9
    scale = np.abs(expect).max()
    assert np.abs(m[cov] - expect[cov]).max() <= 2e-6 * scale
    assert np.all(m[~cov] == 0.0)


def test_linear_face_pressure_gives_linear_vertex_and_map_values():
    """On the uniform Kuhn top of the 1,800-tet pad every interior vertex has a
    point-symmetric fan of six equal triangles, and an in-plane affine map x =
    A X keeps it so.  A face field p_f = a . c_f + b (c_f the deformed face
    centroid) therefore averages to p_v = a . (A X_v) + b at interior vertices,
    and the map shows a . (A X_c) + b at pixels inside faces of interior
    vertices."""
    env = workloads.pad_env(0, steps=1)
    sc = Scene(env)
    A = np.array([[1.08, 0.04, 0.0], [-0.02, 0.95, 0.0], [0.0, 0.0, 1.0]])
    x = sc.X @ A.T
    a, b = np.array([3.0e5, -1.0e5]), 12.0
    f = sc.cfaces
    cent = (x[f[:, 0]] + x[f[:, 1]] + x[f[:, 2]]) / 3.0
    pf = a[0] * cent[:, 0] + a[1] * cent[:, 1] + b
    pv = sc.vertex_pressure(x=x, p_face=pf)
    Xc = sc.X[sc.cverts]
    L = 20e-3
    interior = (Xc[:, 0] > 0) & (Xc[:, 0] < L) & (Xc[:, 1] > 0) & (Xc[:, 1] < L)
    xv = Xc @ A.T
    lin = a[0] * xv[:, 0] + a[1] * xv[:, 1] + b
    assert interior.sum() == 81
    assert np.abs(pv[interior] - lin[interior]).max() <= 1e-9 * np.abs(lin).max()
    assert np.abs(pv[~interior] - lin[~interior]).max() > 1e-3 * np.abs(lin).max()  # boundary fans are one-sided
    m, mask = sc.pressure_map(p_vertex=pv)
    U, Vv = _pixel_centres(env["grid"])
    P = np.stack([U, Vv, np.zeros_like(U)], axis=-1) @ A.T
    expect = a[0] * P[..., 0] + a[1] * P[..., 1] + b
    slot = -np.ones(sc.nv, dtype=np.int64)
    slot[sc.cverts] = np.arange(len(sc.cverts))
    pf_ = sc.pix_face.reshape(mask.shape)
    inner = np.zeros(mask.shape, dtype=bool)
    cov = pf_ >= 0
    inner[cov] = interior[slot[sc.cfaces[pf_[cov]]]].all(axis=1)
    assert inner.sum() > 400
    assert np.abs(m[inner] - expect[inner]).max() <= 2e-6 * np.abs(expect).max()


def test_dynamic_energy_matches_gradient_by_finite_differences():
    """The line search's energy (Scene.energy) and the Newton gradient
    (Scene.gradient_hessian) describe one potential in the dynamic case:
    central differences of the energy along random directions equal g . d,
    and both report the same value, with contact pairs and inertia active."""
    env = workloads.small_env(4, dt=1.0 / 60.0, steps=2)
    sc = Scene(env)
    sc.step(env["poses"][0])
    Y = sc.indenter(env["poses"][1])
    rng = np.random.default_rng(5)
    sc.v = sc.v + 1e-3 * rng.standard_normal(sc.v.shape)
    x_tilde = sc.x + sc.h * sc.v
    x = sc.x.copy()
    E, g, _ = sc.gradient_hessian(x, Y, x_tilde)
    cand = sc.candidates(x, Y)
    assert sum(len(gi) for gi, _ in cand.values()) > 0
    assert sc.energy(x, Y, cand, x_tilde) == pytest.approx(E, rel=1e-12)
    eps = 1e-10
    for _ in range(3):
        d = rng.standard_normal(x.shape)
        d[sc.fixed] = 0.0
        fd = (sc.energy(x + eps * d, Y, cand, x_tilde) - sc.energy(x - eps * d, Y, cand, x_tilde)) / (2 * eps)
        assert fd == pytest.approx(float(np.sum(g * d)), rel=1e-5)


# ----------------------------------------------- Algorithm 2's vertex forces

def test_vertex_contact_forces_sum_rules(stepped):
    """The per-vertex decomposition of Algorithm 2: the forces add up to the
    total contact force, f_n + f_tau = f with f_tau normal to n, the vertex
    areas partition the contact surface's area, the normals are unit and
    outward, and p = |f| / A."""
    _, sc, _ = stepped
    f, fn, ft, p, n, A = sc.vertex_contact_forces()
    assert np.allclose(f.sum(axis=0), sc.contact_force(), rtol=1e-12, atol=1e-15)
    assert np.allclose(fn + ft, f, atol=1e-14 * np.abs(f).max())
    assert np.abs(np.einsum("ki,ki->k", ft, n)).max() <= 1e-12 * np.abs(f).max()
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)
    assert np.all(n[:, 2] > 0.9)
    x = sc.x
    c = np.cross(x[sc.cfaces[:, 1]] - x[sc.cfaces[:, 0]], x[sc.cfaces[:, 2]] - x[sc.cfaces[:, 0]])
    assert A.sum() == pytest.approx(0.5 * np.linalg.norm(c, axis=1).sum(), rel=1e-12)
    assert np.allclose(p * A, np.linalg.norm(f, axis=1), rtol=1e-12)
    # the pressed vertices carry a force into the gel (-z), the others none
    assert f[:, 2].min() < 0 and np.count_nonzero(np.linalg.norm(f, axis=1)) < len(f)


def test_vertex_normal_and_area_worked_example():
    """A hub with two faces: one flat (area 1/2, normal +z) and one tilted by
    45 degrees (area sqrt(2)/2, normal (0, 1, 1)/sqrt(2)).  The hub's area is
    (1/2 + sqrt(2)/2) / 3 and its normal the normalised area-weighted sum
    (0, 0, 1/2) + (0, 1/2, 1/2), i.e. (0, 1, 2) / sqrt(5); the rim vertices
    take their single face's normal and a third of its area."""
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 1]], dtype=np.float64)
    sc = Scene.__new__(Scene)
    sc.x, sc.cfaces = x, np.array([[0, 1, 2], [0, 3, 4]])
    sc.cverts, sc.csr_off, sc.csr_idx = msh.vertex_face_csr(sc.cfaces)
    n, A = sc.vertex_normals_areas()
    assert np.allclose(n[0], np.array([0, 1, 2]) / np.sqrt(5), atol=1e-15)
    assert A[0] == pytest.approx((0.5 + np.sqrt(2) / 2) / 3, rel=1e-15)
    assert np.allclose(n[1], [0, 0, 1]) and np.allclose(n[4], np.array([0, 1, 1]) / np.sqrt(2))
    assert A[2] == pytest.approx(0.5 / 3) and A[3] == pytest.approx(np.sqrt(2) / 6)


# ------------------------------------------------ depth map (Sec. III-D)

def test_depth_map_rest_and_affine():
    """At rest the map is the flat top height everywhere on the pad; under
    x = A X + c with the top tilted (z' = z + a x + b y) and shifted in the
    plane, every covered pixel centre shows the tilted plane's height at the
    point of the rest surface that the map sends there (exact for a plane),
    and pixels off the moved surface are uncovered."""
    env = workloads.pad_env(0, steps=1)
    sc = Scene(env)
    m, mask = sc.depth_map()
    assert mask.all() and np.all(m == np.float32(4e-3))
    A = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [2e-3, -1e-3, 1.0]])
    c = np.array([0.7e-3, -0.4e-3, 0.0])
    x = sc.X @ A.T + c
    m, mask = sc.depth_map(x)
    U, Vv = _pixel_centres(env["grid"])
    Xr, Yr = U - c[0], Vv - c[1]                      # rest point mapped to the pixel centre
    expect = (4e-3 + 2e-3 * Xr - 1e-3 * Yr).astype(np.float32)
    inside = (Xr > 1e-9) & (Xr < 20e-3 - 1e-9) & (Yr > 1e-9) & (Yr < 20e-3 - 1e-9)
    outside = (Xr < -1e-9) | (Xr > 20e-3 + 1e-9) | (Yr < -1e-9) | (Yr > 20e-3 + 1e-9)
    assert np.all(mask[inside] == 1) and np.all(mask[outside] == 0)
    assert np.abs(m[inside] - expect[inside]).max() <= 2 * np.spacing(np.float32(4e-3))


def test_depth_map_takes_the_surface_nearest_the_indenter():
    """Two overlapping faces at different heights over the same pixels (a
    fold): the z-buffer keeps the higher one, whichever comes first."""
    x = np.array([[0, 0, 1.0], [1, 0, 1.0], [0, 1, 1.0], [0, 0, 2.0], [1, 0, 2.0], [0, 1, 2.0]])
    for faces in ([[0, 1, 2], [3, 4, 5]], [[3, 4, 5], [0, 1, 2]]):
        sc = Scene.__new__(Scene)
        sc.cfaces = np.array(faces)
        sc.thick_axis, sc.out_sign = 2, 1.0
        g = dict(axis_u=0, axis_v=1, origin=(0.0, 0.0), pixel=(0.1, 0.1), H=10, W=10)
        m, mask = sc.depth_map(x, grid=g)
        r, c = np.indices((10, 10))
        assert np.all(m[mask == 1] == 2.0)
        assert np.all(mask[r + c <= 8] == 1) and np.all(mask[r + c >= 10] == 0)  # centres on the hypotenuse: either
