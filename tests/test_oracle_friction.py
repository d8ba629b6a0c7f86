"""Pins for oracle/friction.py (IPC lagged friction with the friction ratio
and velocity threshold of Sec. III-B): the smoothed friction function's
closed forms, finite differences of the potential, its gradient and Hessian,
Coulomb's law in the sliding regime (force mu * lambda per pair, opposite to
the relative sliding), the smoothed static regime below the velocity
threshold, no friction from normal motion, and a whole dynamic step with
slip whose tangential force stays within the Coulomb bound."""
import copy

import numpy as np
import pytest

from oracle import friction as fr
from oracle.sim import Scene
from synth import workloads

EX = 1e-4


def test_smoothing_closed_forms():
    """f0(0) = eps_x / 3, f0 and f1 continuous at eps_x with f0 = y, f1 = 1
    beyond it, f1 = f0' (central differences), 0 <= f1 <= 1, f1 / y and the
    curvature coefficient match their definitions."""
    assert fr.f0(0.0, EX) == pytest.approx(EX / 3, rel=1e-15)
    for y in (EX, EX * (1 - 1e-12), EX * (1 + 1e-12)):
        assert fr.f0(y, EX) == pytest.approx(EX, rel=1e-9)
        assert fr.f1(y, EX) == pytest.approx(1.0, rel=1e-9)
    ys = np.linspace(0.01, 3.0, 300) * EX
    h = 1e-7 * EX
    fd = (fr.f0(ys + h, EX) - fr.f0(ys - h, EX)) / (2 * h)
    assert np.allclose(fd, fr.f1(ys, EX), rtol=1e-6, atol=1e-9)
    assert np.all((fr.f1(ys, EX) >= 0) & (fr.f1(ys, EX) <= 1 + 1e-15))
    assert np.allclose(fr.f1_over_y(ys, EX), fr.f1(ys, EX) / ys, rtol=1e-13)
    d1 = (fr.f1(ys + h, EX) - fr.f1(ys - h, EX)) / (2 * h)
    assert np.allclose(fr.curvature(ys, EX), (d1 * ys - fr.f1(ys, EX)) / ys ** 3, rtol=1e-5)
    assert fr.f1_over_y(0.0, EX) == pytest.approx(2 / EX)


@pytest.fixture(scope="module")
def lagged():
    """A small pad pressed by a sphere (one dynamic step), friction lagged at
    the converged state."""
    env = copy.deepcopy(workloads.small_env(4, dt=1.0 / 60.0, steps=1))
    env["opts"]["friction_mu"] = 0.5
    sc = Scene(env)
    sc.step(env["poses"][0])
    Y = sc.indenter(sc.pose)
    pairs = fr.lag(sc, sc.x, Y)
    assert pairs.count() > 5
    return sc, pairs, sc.x.copy(), Y


def _total(sc, pairs, x, x_t, Y, Y_t, need_hess=True):
    return fr.potential(sc, pairs, x, x_t, Y, Y_t, 0.5, EX, need_hess)


def _assemble(sc, terms):
    g = np.zeros(3 * sc.nv)
    H = np.zeros((3 * sc.nv, 3 * sc.nv))
    for gv, gg, HH in terms:
        k = gv.shape[1]
        d = (3 * gv[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 3 * k)
        for r in range(len(gv)):
            np.add.at(g, d[r], gg[r])
            H[np.ix_(d[r], d[r])] += HH[r]
    return g, H


@pytest.mark.parametrize("scale", [0.3, 5.0])
def test_potential_gradient_and_hessian_by_finite_differences(lagged, scale):
    """Below (scale 0.3) and beyond (5) the threshold: central differences of
    D match the gradient, differences of the gradient match the Hessian, and
    the Hessian is PSD."""
    sc, pairs, x0, Y = lagged
    rng = np.random.default_rng(3)
    x = x0 + scale * EX * rng.standard_normal(x0.shape)
    Yt = Y - scale * EX * np.array([1.0, 0.5, 0.0])
    _, terms = _total(sc, pairs, x, x0, Y, Yt)
    g, H = _assemble(sc, terms)
    eps = 1e-6 * EX
    for _ in range(4):
        d = rng.standard_normal(x.shape)
        Dp = _total(sc, pairs, x + eps * d, x0, Y, Yt, False)[0]
        Dm = _total(sc, pairs, x - eps * d, x0, Y, Yt, False)[0]
        assert (Dp - Dm) / (2 * eps) == pytest.approx(float(g @ d.ravel()), rel=1e-5, abs=1e-12)
        gp = _assemble(sc, _total(sc, pairs, x + eps * d, x0, Y, Yt)[1])[0]
        gm = _assemble(sc, _total(sc, pairs, x - eps * d, x0, Y, Yt)[1])[0]
        assert np.allclose((gp - gm) / (2 * eps), H @ d.ravel(), rtol=1e-4, atol=1e-6 * np.abs(H).max() * EX)
    assert np.linalg.eigvalsh(H).min() >= -1e-9 * np.abs(H).max()


def _per_pair_forces(sc, pairs, x, x_t, Y, Y_t):
    """Friction force on the gel per pair: minus the sum of its gel slots'
    gradients."""
    _, terms = _total(sc, pairs, x, x_t, Y, Y_t)
    return np.concatenate([-gg.reshape(len(gv), -1, 3).sum(axis=1) for gv, gg, _ in terms])


def _lams(pairs):
    return np.concatenate([v[4] for v in pairs.data.values()])


def test_sliding_regime_is_coulomb(lagged):
    """Gel held, indenter moved tangentially by 20 eps_x: every pair slides
    and its friction force on the gel has magnitude mu * lambda, pointing
    along the indenter's motion (the indenter drags the gel)."""
    sc, pairs, x0, Y = lagged
    dY = np.array([20 * EX, 0.0, 0.0])
    F = _per_pair_forces(sc, pairs, x0, x0, Y + dY, Y)
    lam = _lams(pairs)
    assert np.allclose(np.linalg.norm(F, axis=1), 0.5 * lam, rtol=1e-9)
    # each force lies in its pair's tangent plane and has a positive x part
    assert np.all(F[:, 0] > 0)
    total = F.sum(axis=0)
    assert total[0] == pytest.approx(0.5 * lam.sum(), rel=0.05)


def test_static_regime_below_threshold(lagged):
    """Sliding 1e-3 eps_x: every pair's force is mu * lambda * f1(y) with
    y ~ 1e-3 eps_x, i.e. about 2e-3 of the Coulomb force (the smoothed static
    regime of the velocity threshold)."""
    sc, pairs, x0, Y = lagged
    dY = np.array([0.0, 1e-3 * EX, 0.0])
    F = _per_pair_forces(sc, pairs, x0, x0, Y + dY, Y)
    ratio = np.linalg.norm(F, axis=1) / (0.5 * _lams(pairs))
    assert np.all(ratio < 2.1e-3) and np.all(ratio > 0)


def test_normal_motion_gives_no_friction(lagged):
    """Each pair moved along its own lagged normal only: zero friction force
    (checked pair by pair through a one-pair lag)."""
    sc, pairs, x0, Y = lagged
    for kind, (gi, ii, w, nrm, lam) in pairs.data.items():
        one = fr.LaggedPairs()
        one.data[kind] = (gi[:1], ii[:1], w[:1], nrm[:1], lam[:1])
        # move every indenter vertex along the pair's normal
        F = _per_pair_forces(sc, one, x0, x0, Y + 50 * EX * nrm[0], Y)
        assert np.abs(F).max() <= 1e-12 * lam[0]


def test_dynamic_step_with_slip_respects_coulomb_bound():
    """A sphere pressed and dragged along x over two dynamic steps with
    friction 0.5: the tangential contact force points along the drag and its
    size stays below mu times the normal force (up to the lag between the
    normal forces of consecutive substeps), well above zero; without
    friction it nearly vanishes."""
    env = copy.deepcopy(workloads.small_env(4, dt=1.0 / 60.0, steps=3))
    for k, p in enumerate(env["poses"]):
        p["t"] = p["t"] + np.array([0.2e-3 * (k + 1), 0.0, 0.0])
    out = {}
    for mu in (0.0, 0.5):
        e = copy.deepcopy(env)
        e["opts"]["friction_mu"] = mu
        sc = Scene(e)
        for p in e["poses"]:
            sc.step(p)
        out[mu] = sc.contact_force()
        assert all(np.all(np.diff(t) <= 0) for t in sc.trace if len(t) > 1)
    f = out[0.5]
    assert f[0] > 0.3 * 0.5 * abs(f[2])
    assert np.hypot(f[0], f[1]) <= 0.5 * abs(f[2]) * 1.05
    assert abs(out[0.0][0]) < 0.1 * f[0]
