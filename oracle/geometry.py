"""Primitive distances, IPC barrier and mollifier (oracle, FP64).

Distance.  For point-triangle (points p, t0, t1, t2) and edge-edge (a0, a1,
b0, b1) pairs the unsigned distance is the minimum, over every pair of faces
(sub-simplices) of the two primitives whose closest points lie strictly inside
both faces, of the distance between the two affine hulls.  Each candidate
writes the difference vector as r = sum_i w_i(beta) x_i with weights affine
in the face parameters beta; beta solves the normal equations.

Derivatives.  With f(x, beta) = |r|^2 minimised over beta on the active faces
(envelope theorem):  grad_i f = 2 w_i r  and
    Hess f = f_xx - f_xb f_bb^-1 f_bx,
    f_xx = 2 (w w^T (x) I3),  f_bb = 2 D^T D,  f_{x_i b_c} = 2 (B_ic r + w_i D_c),
with D_c = sum_i B_ic x_i the direction of parameter c.

Barrier (Li et al. 2020, "Incremental Potential Contact"), on the unsquared
distance d:  b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat, else 0.
Edge-edge mollifier: c = |(a1-a0) x (b1-b0)|^2, eps_x = 1e-3 |a1-a0|_rest^2
|b1-b0|_rest^2, m(c) = (2 - c/eps_x) c/eps_x for c < eps_x, else 1; the
edge-edge barrier is m(c) b(d).
"""
import itertools
import numpy as np

# ------------------------------------------------------------ face candidates

def _faces_of(vertices):
    """All non-empty subsets (faces) of a simplex given by vertex slots."""
    out = []
    for k in range(1, len(vertices) + 1):
        out += list(itertools.combinations(vertices, k))
    return out


def _candidate(face_a, face_b, m=4):
    """(a, B) such that r = sum_i (a_i + sum_c B_ic beta_c) x_i is the vector
    from a point of face_b to a point of face_a."""
    a = np.zeros(m)
    cols = []
    a[face_a[0]] += 1.0
    for v in face_a[1:]:
        col = np.zeros(m)
        col[v], col[face_a[0]] = 1.0, -1.0
        cols.append(col)
    a[face_b[0]] -= 1.0
    for v in face_b[1:]:
        col = np.zeros(m)
        col[v], col[face_b[0]] = -1.0, 1.0
        cols.append(col)
    B = np.stack(cols, axis=1) if cols else np.zeros((m, 0))
    return a, B, len(face_a) - 1


PT_CANDIDATES = [_candidate((0,), fb) for fb in _faces_of((1, 2, 3))]
EE_CANDIDATES = [_candidate(fa, fb) for fa in _faces_of((0, 1)) for fb in _faces_of((2, 3))]


def _solve_candidate(x, a, B, ka):
    """For points x (n,4,3): beta (n,k), feasibility (n,), d^2 (n,)."""
    n = x.shape[0]
    r0 = np.einsum("i,nij->nj", a, x)
    k = B.shape[1]
    if k == 0:
        return np.zeros((n, 0)), np.ones(n, dtype=bool), np.einsum("nj,nj->n", r0, r0)
    D = np.einsum("ic,nij->ncj", B, x)            # (n, k, 3)
    G = np.einsum("ncj,ndj->ncd", D, D)           # (n, k, k)
    rhs = -np.einsum("ncj,nj->nc", D, r0)
    det = np.linalg.det(G)
    scale = np.prod(np.einsum("ncc->nc", G), axis=1)
    ok = det > 1e-20 * np.maximum(scale, 1e-300)
    beta = np.zeros((n, k))
    if np.any(ok):
        beta[ok] = np.linalg.solve(G[ok], rhs[ok][..., None])[..., 0]
    # barycentric coordinates on each face must be strictly positive
    feas = ok.copy()
    ba, bb = beta[:, :ka], beta[:, ka:]
    if ka > 0:
        feas &= np.all(ba > 0, axis=1) & (ba.sum(axis=1) < 1)
    if k - ka > 0:
        feas &= np.all(bb > 0, axis=1) & (bb.sum(axis=1) < 1)
    r = r0 + np.einsum("nc,ncj->nj", beta, D)
    return beta, feas, np.einsum("nj,nj->n", r, r)


def distance_sq(x, kind):
    """Squared distance and index of the active candidate for pairs x (n,4,3);
    kind 'pt' (point, tri) or 'ee' (edge, edge)."""
    cands = PT_CANDIDATES if kind == "pt" else EE_CANDIDATES
    n = x.shape[0]
    best = np.full(n, np.inf)
    which = np.full(n, -1)
    for ci, (a, B, ka) in enumerate(cands):
        _, feas, d2 = _solve_candidate(x, a, B, ka)
        take = feas & (d2 < best)
        best[take] = d2[take]
        which[take] = ci
    return best, which


def distance_sq_derivatives(x, kind):
    """d^2, its gradient (n,12) and Hessian (n,12,12) on the active faces."""
    cands = PT_CANDIDATES if kind == "pt" else EE_CANDIDATES
    d2, which = distance_sq(x, kind)
    n = x.shape[0]
    g = np.zeros((n, 12))
    H = np.zeros((n, 12, 12))
    I3 = np.eye(3)
    for ci, (a, B, ka) in enumerate(cands):
        sel = np.nonzero(which == ci)[0]
        if len(sel) == 0:
            continue
        xs = x[sel]
        beta, _, _ = _solve_candidate(xs, a, B, ka)
        w = a[None, :] + beta @ B.T                     # (s, 4)
        r = np.einsum("ni,nij->nj", w, xs)              # (s, 3)
        g[sel] = (2.0 * w[:, :, None] * r[:, None, :]).reshape(-1, 12)
        Hxx = 2.0 * np.einsum("ni,nl,jk->nijlk", w, w, I3).reshape(-1, 12, 12)
        k = B.shape[1]
        if k > 0:
            D = np.einsum("ic,nij->ncj", B, xs)
            Fxb = 2.0 * (np.einsum("ic,nj->nijc", B, r) + np.einsum("ni,ncj->nijc", w, D))
            Fxb = Fxb.reshape(-1, 12, k)
            Fbb = 2.0 * np.einsum("ncj,ndj->ncd", D, D)
            Hxx = Hxx - Fxb @ np.linalg.solve(Fbb, np.swapaxes(Fxb, 1, 2))
        H[sel] = Hxx
    return d2, g, H


# ------------------------------------------------------------------- barrier

def barrier(d, dhat):
    """b, b', b'' of the IPC log barrier on the unsquared distance."""
    d = np.asarray(d, dtype=np.float64)
    inside = (d > 0) & (d < dhat)
    dd = np.where(inside, d, dhat)
    L = np.log(dd / dhat)
    e = dd - dhat
    with np.errstate(over="ignore", divide="ignore"):
        b = np.where(inside, -e * e * L, 0.0)
        b1 = np.where(inside, -2.0 * e * L - e * e / dd, 0.0)
        b2 = np.where(inside, -2.0 * L - 4.0 * e / dd + e * e / (dd * dd), 0.0)
    return b, b1, b2


def barrier_derivatives(d2, g2, H2, dhat):
    """b(d(x)) with gradient and Hessian from those of d^2 (chain rule)."""
    d = np.sqrt(d2)
    b, b1, b2 = barrier(d, dhat)
    gd = g2 / (2.0 * d)[:, None]
    Hd = H2 / (2.0 * d)[:, None, None] - np.einsum("ni,nj->nij", g2, g2) / (4.0 * d ** 3)[:, None, None]
    gb = b1[:, None] * gd
    Hb = b2[:, None, None] * np.einsum("ni,nj->nij", gd, gd) + b1[:, None, None] * Hd
    return b, gb, Hb


def cross_sq(x):
    """c = |(a1-a0) x (b1-b0)|^2 with gradient (n,12) and Hessian (n,12,12)."""
    u = x[:, 1] - x[:, 0]
    v = x[:, 3] - x[:, 2]
    uu = np.einsum("ni,ni->n", u, u)
    vv = np.einsum("ni,ni->n", v, v)
    uv = np.einsum("ni,ni->n", u, v)
    c = uu * vv - uv * uv
    gu = 2.0 * vv[:, None] * u - 2.0 * uv[:, None] * v
    gv = 2.0 * uu[:, None] * v - 2.0 * uv[:, None] * u
    I3 = np.eye(3)
    Huu = 2.0 * vv[:, None, None] * I3 - 2.0 * np.einsum("ni,nj->nij", v, v)
    Hvv = 2.0 * uu[:, None, None] * I3 - 2.0 * np.einsum("ni,nj->nij", u, u)
    Huv = 4.0 * np.einsum("ni,nj->nij", u, v) - 2.0 * np.einsum("ni,nj->nij", v, u) - 2.0 * uv[:, None, None] * I3
    # map (u, v) -> points: u = x1 - x0, v = x3 - x2
    Su = np.array([-1.0, 1.0, 0.0, 0.0])
    Sv = np.array([0.0, 0.0, -1.0, 1.0])
    g = (Su[None, :, None] * gu[:, None, :] + Sv[None, :, None] * gv[:, None, :]).reshape(-1, 12)
    H = (np.einsum("a,b,nij->naibj", Su, Su, Huu) + np.einsum("a,b,nij->naibj", Sv, Sv, Hvv)
         + np.einsum("a,b,nij->naibj", Su, Sv, Huv) + np.einsum("a,b,nji->naibj", Sv, Su, Huv))
    return c, g, H.reshape(-1, 12, 12)


def mollifier(c, eps_x):
    t = c / eps_x
    inside = t < 1.0
    m = np.where(inside, (2.0 - t) * t, 1.0)
    m1 = np.where(inside, (2.0 - 2.0 * t) / eps_x, 0.0)
    m2 = np.where(inside, -2.0 / (eps_x * eps_x), 0.0)
    return m, m1, m2


def pair_barrier(x, kind, dhat, eps_x=None, need_hess=True):
    """Energy b (n,), gradient (n,12), Hessian (n,12,12) of one pair type.
    For 'ee', eps_x (n,) enables the mollifier m(c) b(d)."""
    if need_hess:
        d2, g2, H2 = distance_sq_derivatives(x, kind)
        b, gb, Hb = barrier_derivatives(d2, g2, H2, dhat)
    else:
        d2, _ = distance_sq(x, kind)
        b = barrier(np.sqrt(d2), dhat)[0]
        return b, None, None
    if kind == "ee" and eps_x is not None:
        c, gc, Hc = cross_sq(x)
        m, m1, m2 = mollifier(c, eps_x)
        gm = m1[:, None] * gc
        Hm = m2[:, None, None] * np.einsum("ni,nj->nij", gc, gc) + m1[:, None, None] * Hc
        H = (b[:, None, None] * Hm + np.einsum("ni,nj->nij", gm, gb)
             + np.einsum("ni,nj->nij", gb, gm) + m[:, None, None] * Hb)
        g = b[:, None] * gm + m[:, None] * gb
        return m * b, g, H
    return b, gb, Hb


def ee_energy_only(x, dhat, eps_x):
    d2, _ = distance_sq(x, "ee")
    b = barrier(np.sqrt(d2), dhat)[0]
    u = x[:, 1] - x[:, 0]
    v = x[:, 3] - x[:, 2]
    c = np.einsum("ni,ni->n", np.cross(u, v), np.cross(u, v))
    return mollifier(c, eps_x)[0] * b
