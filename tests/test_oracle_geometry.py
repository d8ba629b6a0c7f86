"""Pins for oracle/geometry.py and oracle/ccd.py: distances against textbook
special cases and dense brute-force sampling, derivatives against central
finite differences, barrier and mollifier identities, and the conservative
time of impact of additive CCD against exact impact times."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle.ccd import accd


def _sample_pt(x, n=301):
    """min over a dense barycentric grid of |p - t(b)|."""
    p, a, b, c = x
    s = np.linspace(0, 1, n)
    S, T = np.meshgrid(s, s)
    m = S + T <= 1
    pts = a + S[m][:, None] * (b - a) + T[m][:, None] * (c - a)
    return np.sqrt(((pts - p) ** 2).sum(axis=1).min())


def _sample_ee(x, n=401):
    a0, a1, b0, b1 = x
    s = np.linspace(0, 1, n)
    A = a0 + s[:, None] * (a1 - a0)
    B = b0 + s[:, None] * (b1 - b0)
    return np.sqrt(((A[:, None, :] - B[None, :, :]) ** 2).sum(axis=2).min())


def test_pt_special_cases():
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    cases = [((0.2, 0.2, 0.5), 0.5),                 # above the interior: height
             ((-1.0, -1.0, 0.0), np.sqrt(2.0)),      # vertex region
             ((0.5, -2.0, 0.0), 2.0),                # edge region
             ((1.0, 1.0, 1.0), np.sqrt(0.5 + 1.0))]  # hypotenuse edge region
    for p, d in cases:
        x = np.concatenate([np.array(p)[None], tri])[None]
        d2, _ = geo.distance_sq(x, "pt")
        assert np.sqrt(d2[0]) == pytest.approx(d, rel=1e-12)


def test_ee_special_cases():
    # skew perpendicular segments crossing above each other at height 1
    x = np.array([[[-1, 0, 0], [1, 0, 0], [0, -1, 1], [0, 1, 1]]], dtype=float)
    assert np.sqrt(geo.distance_sq(x, "ee")[0][0]) == pytest.approx(1.0, rel=1e-12)
    # parallel overlapping segments at distance 0.5
    x = np.array([[[0, 0, 0], [2, 0, 0], [1, 0.5, 0], [3, 0.5, 0]]], dtype=float)
    assert np.sqrt(geo.distance_sq(x, "ee")[0][0]) == pytest.approx(0.5, rel=1e-12)
    # endpoint-endpoint
    x = np.array([[[0, 0, 0], [1, 0, 0], [2, 1, 0], [3, 1, 0]]], dtype=float)
    assert np.sqrt(geo.distance_sq(x, "ee")[0][0]) == pytest.approx(np.sqrt(2.0), rel=1e-12)


def test_distance_vs_sampling():
    rng = np.random.default_rng(0)
    for _ in range(30):
        x = rng.standard_normal((4, 3))
        d = np.sqrt(geo.distance_sq(x[None], "pt")[0][0])
        ds = _sample_pt(x)
        assert d <= ds + 1e-12 and ds - d < 2e-2
        d = np.sqrt(geo.distance_sq(x[None], "ee")[0][0])
        ds = _sample_ee(x)
        assert d <= ds + 1e-12 and ds - d < 1e-2


def _fd_check(f, x, h=1e-6, rtol=1e-5):
    """Central differences of scalar f at x (12,)."""
    g = np.zeros(12)
    for i in range(12):
        e = np.zeros(12)
        e[i] = h
        g[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


@pytest.mark.parametrize("kind", ["pt", "ee"])
def test_distance_derivatives_fd(kind):
    rng = np.random.default_rng(1 if kind == "pt" else 2)
    n_ok = 0
    for _ in range(40):
        x = rng.standard_normal((1, 4, 3))
        d2, g, H = geo.distance_sq_derivatives(x, kind)
        # skip configurations near a region switch (FD would straddle it)
        d2p, wp = geo.distance_sq(x + 1e-4 * rng.standard_normal(x.shape), kind)
        if wp[0] != geo.distance_sq(x, kind)[1][0]:
            continue
        n_ok += 1
        f = lambda v: geo.distance_sq(v.reshape(1, 4, 3), kind)[0][0]
        gf = _fd_check(f, x.ravel())
        assert np.allclose(gf, g[0], rtol=1e-5, atol=1e-7)
        Hf = np.stack([_fd_check(lambda v, i=i: geo.distance_sq_derivatives(v.reshape(1, 4, 3), kind)[1][0, i], x.ravel())
                       for i in range(12)])
        assert np.allclose(Hf, H[0], rtol=1e-4, atol=1e-6)
    assert n_ok > 20


def test_barrier_identities():
    dhat = 1e-3
    d = np.array([dhat, 2 * dhat, 0.5 * dhat])
    b, b1, b2 = geo.barrier(d, dhat)
    assert b[0] == 0 and b1[0] == 0 and b[1] == 0
    # C1 at dhat, positive and decreasing inside
    assert b[2] > 0 and b1[2] < 0 and b2[2] > 0
    small = geo.barrier(np.array([1e-6, 1e-9, 1e-200]), dhat)[0]
    assert b[2] < small[0] < small[1] < small[2] and small[2] > 1e3 * b[2]
    # derivatives by central differences
    dd = np.linspace(0.05, 0.95, 19) * dhat
    h = 1e-9
    bp = (geo.barrier(dd + h, dhat)[0] - geo.barrier(dd - h, dhat)[0]) / (2 * h)
    bpp = (geo.barrier(dd + h, dhat)[1] - geo.barrier(dd - h, dhat)[1]) / (2 * h)
    _, b1, b2 = geo.barrier(dd, dhat)
    assert np.allclose(bp, b1, rtol=1e-6)
    assert np.allclose(bpp, b2, rtol=1e-5)


def test_mollifier_is_c1():
    eps = 0.3
    m, m1, _ = geo.mollifier(np.array([eps * (1 - 1e-12), eps, 0.0]), eps)
    assert m[0] == pytest.approx(1.0) and m[1] == 1.0 and m[2] == 0.0
    assert abs(m1[0]) < 1e-9


@pytest.mark.parametrize("kind", ["pt", "ee"])
def test_pair_barrier_fd(kind):
    rng = np.random.default_rng(3)
    dhat = 0.5
    tested = 0
    for _ in range(200):
        x = rng.standard_normal((1, 4, 3))
        d = np.sqrt(geo.distance_sq(x, kind)[0][0])
        if not (0.1 < d < 0.45):
            continue
        if geo.distance_sq(x + 1e-4 * rng.standard_normal(x.shape), kind)[1][0] != geo.distance_sq(x, kind)[1][0]:
            continue
        eps = np.array([5.0]) if kind == "ee" else None  # mollifier active
        b, g, H = geo.pair_barrier(x, kind, dhat, eps)
        f = lambda v: geo.pair_barrier(v.reshape(1, 4, 3), kind, dhat, eps)[0][0]
        assert np.allclose(_fd_check(f, x.ravel()), g[0], rtol=1e-5, atol=1e-8)
        Hf = np.stack([_fd_check(lambda v, i=i: geo.pair_barrier(v.reshape(1, 4, 3), kind, dhat, eps)[1][0, i], x.ravel())
                       for i in range(12)])
        assert np.allclose(Hf, H[0], rtol=1e-4, atol=1e-6)
        tested += 1
        if tested >= 6:
            break
    assert tested >= 3


def test_cross_sq_fd():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 4, 3))
    c, g, H = geo.cross_sq(x)
    u, v = x[0, 1] - x[0, 0], x[0, 3] - x[0, 2]
    assert c[0] == pytest.approx(np.sum(np.cross(u, v) ** 2))
    f = lambda w: geo.cross_sq(w.reshape(1, 4, 3))[0][0]
    assert np.allclose(_fd_check(f, x.ravel()), g[0], rtol=1e-6, atol=1e-8)
    Hf = np.stack([_fd_check(lambda w, i=i: geo.cross_sq(w.reshape(1, 4, 3))[1][0, i], x.ravel()) for i in range(12)])
    assert np.allclose(Hf, H[0], rtol=1e-5, atol=1e-6)


def test_accd_point_falling_on_triangle():
    tri = np.array([[-1, -1, 0], [2, -1, 0], [-1, 2, 0]], dtype=float)
    x0 = np.concatenate([np.array([[0.1, 0.1, 1.0]]), tri])[None]
    p = np.zeros_like(x0)
    p[0, 0, 2] = -2.0             # true impact at t = 0.5
    t = accd(x0, p, "pt")[0]
    assert 0.0 < t <= 0.5
    zt = 1.0 - 2.0 * t
    assert zt >= 0.1 * 1.0 - 1e-12          # distance kept >= s * d0
    assert t > 0.5 * (1 - 0.1) - 1e-3      # and not overly timid
    # moving away / missing: no impact before t = 1
    p[0, 0, 2] = +2.0
    assert accd(x0, p, "pt")[0] >= 1.0
    p[0, 0] = [0.0, 0.0, -0.5]
    assert accd(x0, p, "pt")[0] >= 1.0


def test_accd_edges_crossing_and_conservative():
    rng = np.random.default_rng(5)
    x0 = np.array([[[-1, 0, 0], [1, 0, 0], [0, -1, 1], [0, 1, 1]]], dtype=float)
    p = np.zeros_like(x0)
    p[0, 2:, 2] = -1.5            # edge b drops onto edge a at t = 2/3
    t = accd(x0, p, "ee")[0]
    assert 0 < t <= 2.0 / 3.0
    d = np.sqrt(geo.distance_sq(x0 + t * p, "ee")[0][0])
    assert d >= 0.1 - 1e-12
    # random motions: the configuration at the reported time is never closer
    # than s * d0, and neither is any configuration before it
    for _ in range(20):
        x0 = rng.standard_normal((1, 4, 3))
        p = 2 * rng.standard_normal((1, 4, 3))
        t = min(accd(x0, p, "pt")[0], 1.0)
        d0 = np.sqrt(geo.distance_sq(x0, "pt")[0][0])
        for tau in np.linspace(0, t, 25):
            assert np.sqrt(geo.distance_sq(x0 + tau * p, "pt")[0][0]) >= 0.1 * d0 * (1 - 1e-9) - 1e-12 or tau == 0
