"""IPC lagged friction (oracle, FP64) -- TEST INFRASTRUCTURE ONLY.

The paper configures UIPC with a friction ratio of 0.5 and a velocity
threshold of 0.01 m/s (Sec. III-B); UIPC's friction is the lagged, smoothed
Coulomb friction of incremental potential contact (Li et al. 2020, Sec. 5).
Written here from that method:

* Lagging.  At the start of each indenter substep (the converged state of the
  previous substep, or of the previous step), every contact pair with
  d < dhat fixes its normal force magnitude lambda = kappa * m(c) * (-b'(d))
  (m = 1 for point-triangle pairs), the unit normal n of its closest-point
  vector r = sum_i w_i x_i, and the closest-point weights w (r's weights on
  the pair's four points).
* Sliding.  The relative displacement of the closest points since the step
  start, rel = sum_i w_i (x_i - x_i^t) (gel points move with the unknowns,
  indenter points with the kinematic pose), projected on the lagged tangent
  plane: u = P rel, P = I - n n^T, y = |u|.
* Potential.  D(x) = sum_k mu lambda_k f0(y_k) with the C1 smoothing of the
  velocity threshold, eps_x = eps_v * h:
      f0(y) = -y^3 / (3 eps_x^2) + y^2 / eps_x + eps_x / 3   (y < eps_x), y otherwise,
      f1(y) = f0'(y) = 2 y / eps_x - y^2 / eps_x^2           (y < eps_x), 1 otherwise.
  It is added to the incremental potential of the dynamic step (the potential
  divided by h^2, so D is in the units of the elastic energy and its gradient
  is the friction force: magnitude mu lambda when sliding faster than eps_v).
* Derivatives.  With respect to rel: grad = mu lambda (f1(y) / y) u, and
  Hess = mu lambda [ (f1 / y) P + (f1' y - f1) / y^3 u u^T ], which is PSD:
  its eigenvalues are f1' >= 0 along u, f1 / y >= 0 across u in the tangent
  plane, 0 along n.  At y = 0 the limit is (2 / eps_x) P.  A gel point i of
  the pair gets w_i times the gradient, and the block (i, j) w_i w_j Hess.
Friction acts only in dynamic scenes (eps_x needs the time step).
"""
import numpy as np

from . import geometry as geo


def f0(y, ex):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < ex, -y ** 3 / (3 * ex * ex) + y * y / ex + ex / 3, y)


def f1(y, ex):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < ex, 2 * y / ex - y * y / (ex * ex), 1.0)


def f1_over_y(y, ex):
    y = np.asarray(y, dtype=np.float64)
    safe = np.where(y > 0, y, 1.0)
    return np.where(y < ex, 2 / ex - y / (ex * ex), 1.0 / safe)


def curvature(y, ex):
    """(f1'(y) y - f1(y)) / y^3, the coefficient of u u^T (bounded times
    u u^T as y -> 0: -1/(y eps_x^2) below eps_x)."""
    y = np.asarray(y, dtype=np.float64)
    safe = np.where(y > 0, y, 1.0)
    return np.where(y < ex, -1.0 / (safe * ex * ex), -1.0 / safe ** 3)


def closest_weights(x, kind):
    """Closest-point weights w (n, 4) with r = sum_i w_i x_i the vector from
    the closest point of the second primitive to that of the first (the
    active candidate of the oracle's distance), and r itself."""
    cands = geo.PT_CANDIDATES if kind == "pt" else geo.EE_CANDIDATES
    _, which = geo.distance_sq(x, kind)
    n = x.shape[0]
    w = np.zeros((n, 4))
    for ci, (a, B, ka) in enumerate(cands):
        sel = np.nonzero(which == ci)[0]
        if len(sel) == 0:
            continue
        beta, _, _ = geo._solve_candidate(x[sel], a, B, ka)
        w[sel] = a[None, :] + beta @ B.T
    r = np.einsum("ni,nij->nj", w, x)
    return w, r


class LaggedPairs:
    """The lagged friction data of one Newton solve: per pair kind, the gel
    and indenter primitive ids, the weights w (n, 4), unit normals n (n, 3)
    and normal force magnitudes lam (n,)."""

    def __init__(self):
        self.data = {}

    def count(self):
        return sum(len(v[0]) for v in self.data.values())


def lag(scene, x, Y):
    """Contact pairs within dhat at state (x, Y) and their lagged friction
    data (normal force, normal, closest-point weights)."""
    out = LaggedPairs()
    cand = scene.candidates(x, Y)
    for kind, (gi, ii) in cand.items():
        if len(gi) == 0:
            continue
        pts = scene.pair_points(kind, gi, ii, x, Y)
        gk = "ee" if kind == "ee" else "pt"
        d2, _ = geo.distance_sq(pts, gk)
        d = np.sqrt(d2)
        act = (d < scene.dhat) & (d > 0)
        if not np.any(act):
            continue
        gi, ii, pts, d = gi[act], ii[act], pts[act], d[act]
        _, b1, _ = geo.barrier(d, scene.dhat)
        lam = scene.kappa * (-b1)
        if kind == "ee":
            c, _, _ = geo.cross_sq(pts)
            m, _, _ = geo.mollifier(c, scene.eps_x(gi, ii))
            lam = lam * m
        w, r = closest_weights(pts, gk)
        nrm = r / np.linalg.norm(r, axis=1, keepdims=True)
        out.data[kind] = (gi, ii, w, nrm, lam)
    return out


def potential(scene, pairs, x, x_t, Y, Y_t, mu, ex, need_hess=True):
    """D(x) and, with need_hess, the per-pair (gel vertex ids, gradient,
    Hessian) terms in the layout of Scene.barrier_terms."""
    from .sim import GEL_SLOTS
    total = 0.0
    terms = []
    for kind, (gi, ii, w, nrm, lam) in pairs.data.items():
        dx = scene.pair_points(kind, gi, ii, x - x_t, Y - Y_t)       # per-slot displacement since the step start
        rel = np.einsum("ni,nij->nj", w, dx)
        u = rel - np.einsum("nj,nj->n", rel, nrm)[:, None] * nrm
        y = np.linalg.norm(u, axis=1)
        total += float(np.sum(mu * lam * f0(y, ex)))
        if not need_hess:
            continue
        a = mu * lam * f1_over_y(y, ex)
        grel = a[:, None] * u                                          # gradient w.r.t. rel
        P = np.eye(3)[None] - np.einsum("ni,nj->nij", nrm, nrm)
        Hrel = a[:, None, None] * P + (mu * lam * curvature(y, ex))[:, None, None] * np.einsum("ni,nj->nij", u, u)
        slots = GEL_SLOTS[kind]
        ws = w[:, slots]                                               # (n, k)
        k = len(slots)
        g = (ws[:, :, None] * grel[:, None, :]).reshape(-1, 3 * k)
        H = np.einsum("na,nb,nij->naibj", ws, ws, Hrel).reshape(-1, 3 * k, 3 * k)
        gv = scene.pair_gel_vertices(kind, gi)[:, slots]
        terms.append((gv, g, H))
    return total, terms
