"""One implicit step of a tetrahedral gel pad under incremental-potential
contact with a rigid indenter, then stress extraction (oracle, FP64).

Algorithm 2 of the paper: x_{t+1} <- step(x_t, dt); sigma per tet; traction,
normal pressure and tangential traction per surface triangle; contact force
f_k = -g_k / dt^2 from the contact gradient.  The step follows the
incremental potential of Li et al. 2020 with the settings of Sec. III-B
(barrier distance dhat, at most 1024 Newton iterations per step):

  E(x) = 1/(2 h^2) |x - x_tilde|_M^2 + sum_e V_e Psi(F_e) + kappa sum_k b(d_k)
         (dynamic, x_tilde = x_t + h v_t; the whole potential divided by h^2,
          so the contact part of the gradient is the contact force directly)
  E(x) = sum_e V_e Psi(F_e) + kappa sum_k b(d_k)          (quasi-static)

Readings where the paper is silent (each listed in the design notes):
  * kappa <= 0 selects kappa = E * (mean rest length of contact-surface edges).
  * Contact pairs: gel contact-surface vertex vs indenter triangle, indenter
    vertex vs gel contact triangle, gel contact edge vs indenter edge, every
    pair with d < dhat (brute force here).
  * The indenter is kinematic: within one step it moves from its current to
    its target pose in substeps s in [0, 1]; each substep advances s as far as
    additive CCD allows against the current gel (vertex positions linear in s)
    and then solves E for the gel at that indenter pose.
  * Newton: p = -H^-1 g on free DOFs (elastic 9x9 tangent and each pair's
    gel block projected to PSD), alpha_0 = min(1, CCD TOI), halve until
    E(x + alpha p) <= E(x), at most 60 halvings.  Converged when
    |g| <= max(rtol |g_0|, 1e-12 E L^2) or when |p|_inf <= 1e-4 dhat (the step
    is then taken without the energy test); g_0 is the substep's first
    gradient; at most newton_max iterations.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import material as mat
from . import mesh as msh
from . import geometry as geo
from . import friction as fric
from .ccd import accd


# point slots that belong to the gel in each pair type
GEL_SLOTS = {"ptg": [0], "pti": [1, 2, 3], "ee": [0, 1]}


class SimError(RuntimeError):
    pass


class InitialPenetration(SimError):
    pass


class NewtonMaxIter(SimError):
    pass


class LineSearchFail(SimError):
    pass


def _aabb(pts):
    """pts (n, k, 3) -> lo, hi (n, 3)."""
    return pts.min(axis=1), pts.max(axis=1)


def _overlap_pairs(lo1, hi1, lo2, hi2, pad, chunk=2048):
    """All (i, j) with boxes i of set 1 and j of set 2 within ``pad``."""
    out_i, out_j = [], []
    for s in range(0, len(lo1), chunk):
        a_lo, a_hi = lo1[s:s + chunk], hi1[s:s + chunk]
        ok = np.ones((len(a_lo), len(lo2)), dtype=bool)
        for k in range(3):
            ok &= (a_lo[:, None, k] <= hi2[None, :, k] + pad) & (lo2[None, :, k] <= a_hi[:, None, k] + pad)
        i, j = np.nonzero(ok)
        out_i.append(i + s)
        out_j.append(j)
    if not out_i:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    return np.concatenate(out_i), np.concatenate(out_j)


class Scene:
    """Oracle scene: setup (row a0), step (a1-a9), extraction (a10-a14)."""

    def __init__(self, env):
        X = np.asarray(env["X"], dtype=np.float64)
        T = np.asarray(env["tets"], dtype=np.int64)
        m, o = env["material"], env["opts"]
        self.X, self.T = X, T
        self.nv, self.nt = X.shape[0], T.shape[0]
        self.E, self.nu, self.rho = m["E"], m["nu"], m["density"]
        # material law: "snh" (the rest-stable reading, default) or "snh_log"
        # (the full stable Neo-Hookean with its log term)
        self.law = m.get("model", "snh")
        if self.law not in mat.LAWS:
            raise ValueError(f"unknown material law {self.law!r}")
        _, self._psi, self._pk1, self._dpk1, self._cauchy = mat.LAWS[self.law]
        self.mu, self.lam = mat.lame(self.E, self.nu)
        _, self.lam_hat, self.alpha = mat.snh_params(self.E, self.nu)
        self.mp = mat.law_params(self.law, self.E, self.nu)
        if m.get("per_tet") is not None:
            # heterogeneous material: (E, nu) per tet, Eq. 1 and the law's
            # parameters per tet (the scene's E still sets the default kappa)
            pt = np.asarray(m["per_tet"], dtype=np.float64).reshape(-1, 2)
            self.mu, self.lam = mat.lame(pt[:, 0], pt[:, 1])
            _, self.lam_hat, self.alpha = mat.snh_params(pt[:, 0], pt[:, 1])
            self.mp = mat.law_params(self.law, pt[:, 0], pt[:, 1])
        self.Dminv, self.vol = msh.rest_shape(X, T)
        self.Dfx = msh.dF_dx(self.Dminv)
        self.h = float(o["dt"])
        self.dynamic = self.h > 0
        self.mass = msh.lumped_mass(T, self.vol, self.rho, self.nv) if self.dynamic else None
        self.fixed = np.asarray(env["fixed"], dtype=np.int64)
        self.free = np.ones(self.nv, dtype=bool)
        self.free[self.fixed] = False
        # Algorithm 1, steps 1-3
        self.faces, self.parent = msh.boundary_faces(T)
        self.band = msh.contact_band(X, self.fixed, o.get("contact_axis", -1))
        # outward direction of the contact side along the thickness axis
        self.thick_axis = msh.thickness_axis(X, o.get("contact_axis", -1))
        mid = 0.5 * (X[:, self.thick_axis].min() + X[:, self.thick_axis].max())
        self.out_sign = 1.0 if (len(self.fixed) == 0 or X[self.fixed, self.thick_axis].mean() <= mid) else -1.0
        self.cface_ids = msh.contact_faces(self.faces, self.band)
        self.cfaces = self.faces[self.cface_ids].astype(np.int64)
        self.cparent = self.parent[self.cface_ids].astype(np.int64)
        self.cedges = msh.surface_edges(self.cfaces).astype(np.int64)
        self.cverts, self.csr_off, self.csr_idx = msh.vertex_face_csr(self.cfaces)
        self.cverts = self.cverts.astype(np.int64)
        # indenter
        self.ind_V = np.asarray(env["ind_V"], dtype=np.float64)
        self.ind_F = np.asarray(env["ind_F"], dtype=np.int64)
        self.ind_E = msh.surface_edges(self.ind_F).astype(np.int64)
        self.dhat = float(o["dhat"])
        kappa = float(o.get("kappa", 0.0))
        if kappa <= 0:
            el = np.linalg.norm(X[self.cedges[:, 0]] - X[self.cedges[:, 1]], axis=1)
            kappa = self.E * el.mean()
        self.kappa = kappa
        self.gel_elen2 = np.sum((X[self.cedges[:, 0]] - X[self.cedges[:, 1]]) ** 2, axis=1)
        self.ind_elen2 = np.sum((self.ind_V[self.ind_E[:, 0]] - self.ind_V[self.ind_E[:, 1]]) ** 2, axis=1)
        self.rtol = float(o.get("newton_rtol", 1e-6))
        self.newton_max = int(o.get("newton_max", 1024))
        L = np.linalg.norm(X.max(axis=0) - X.min(axis=0))
        self.gabs = 1e-12 * self.E * L * L
        self.ptol = 1e-4 * self.dhat
        self.max_substeps = 256
        # lagged friction (dynamic scenes only): friction ratio and velocity threshold
        self.mu_f = float(o.get("friction_mu", 0.0))
        self.eps_v = float(o.get("friction_eps_v", 0.01))
        self.friction = self.dynamic and self.mu_f > 0
        self._fric = None     # (lagged pairs, x at the step start, indenter at the step start)
        # state
        self.x = X.copy()
        self.v = np.zeros_like(X)
        self.pose = env["start_pose"]
        self.stats = dict(newton=0, substeps=0, steps=0)
        self.trace = []  # per Newton solve: energy at every iterate
        self.grid = env.get("grid")
        if self.grid is not None:
            self.pix_face, self.pix_w = msh.bin_pixels(X, self.cfaces, self.grid)
        if not self.separated(self.x, self.indenter(self.pose)):
            raise InitialPenetration("indenter intersects or touches the gel")

    # ------------------------------------------------------------ geometry
    def indenter(self, pose):
        return self.ind_V @ np.asarray(pose["R"]).T + np.asarray(pose["t"])

    def _gel_prims(self, x):
        return (x[self.cverts][:, None, :], x[self.cedges], x[self.cfaces])

    def _ind_prims(self, Y):
        return (Y[:, None, :], Y[self.ind_E], Y[self.ind_F])

    def candidates(self, x0, Y0, x1=None, Y1=None, pad=None):
        """Brute-force pair lists whose (swept) boxes come within pad."""
        pad = self.dhat if pad is None else pad
        g0, i0 = self._gel_prims(x0), self._ind_prims(Y0)
        g1 = self._gel_prims(x1) if x1 is not None else g0
        i1 = self._ind_prims(Y1) if Y1 is not None else i0

        def box(a, b):
            lo_a, hi_a = _aabb(a)
            lo_b, hi_b = _aabb(b)
            return np.minimum(lo_a, lo_b), np.maximum(hi_a, hi_b)
        gv, ge, gf = (box(a, b) for a, b in zip(g0, g1))
        iv, ie, if_ = (box(a, b) for a, b in zip(i0, i1))
        return dict(ptg=_overlap_pairs(*gv, *if_, pad),
                    pti=_overlap_pairs(*gf, *iv, pad),
                    ee=_overlap_pairs(*ge, *ie, pad))

    def pair_points(self, kind, gi, ii, x, Y):
        if kind == "ptg":
            return np.stack([x[self.cverts[gi]], Y[self.ind_F[ii, 0]], Y[self.ind_F[ii, 1]], Y[self.ind_F[ii, 2]]], axis=1)
        if kind == "pti":
            f = self.cfaces[gi]
            return np.stack([Y[ii], x[f[:, 0]], x[f[:, 1]], x[f[:, 2]]], axis=1)
        e = self.cedges[gi]
        k = self.ind_E[ii]
        return np.stack([x[e[:, 0]], x[e[:, 1]], Y[k[:, 0]], Y[k[:, 1]]], axis=1)

    def pair_gel_vertices(self, kind, gi):
        """(n, 4) gel vertex id per point slot, -1 for indenter slots."""
        n = len(gi)
        out = -np.ones((n, 4), dtype=np.int64)
        if kind == "ptg":
            out[:, 0] = self.cverts[gi]
        elif kind == "pti":
            out[:, 1:] = self.cfaces[gi]
        else:
            out[:, :2] = self.cedges[gi]
        return out

    def eps_x(self, gi, ii):
        return 1e-3 * self.gel_elen2[gi] * self.ind_elen2[ii]

    def min_distance(self, x, Y, cand=None):
        cand = self.candidates(x, Y) if cand is None else cand
        dmin = np.inf
        for kind, (gi, ii) in cand.items():
            if len(gi):
                d2, _ = geo.distance_sq(self.pair_points(kind, gi, ii, x, Y), "pt" if kind != "ee" else "ee")
                dmin = min(dmin, float(np.sqrt(d2.min())))
        return dmin

    def separated(self, x, Y):
        """No pair closer than zero and no gel edge crossing an indenter
        triangle (or the reverse) within the candidate boxes."""
        if self.min_distance(x, Y) <= 0.0:
            return False
        gel_e, ind_f = x[self.cedges], Y[self.ind_F]
        ind_e, gel_f = Y[self.ind_E], x[self.cfaces]
        for E_, F_ in ((gel_e, ind_f), (ind_e, gel_f)):
            lo_e, hi_e = _aabb(E_)
            lo_f, hi_f = _aabb(F_)
            i, j = _overlap_pairs(lo_e, hi_e, lo_f, hi_f, 0.0)
            if len(i) and np.any(_segment_hits_triangle(E_[i], F_[j])):
                return False
        return True

    # ------------------------------------------------------------- energy
    def elastic(self, x, need_hess=True):
        F = msh.deformation_gradient(x, self.T, self.Dminv)
        psi = self._psi(F, *self.mp)
        Ee = float(np.sum(self.vol * psi))
        if not need_hess:
            return Ee, None, None
        P = self._pk1(F, *self.mp).reshape(-1, 9)
        ge = self.vol[:, None] * np.einsum("nki,nk->ni", self.Dfx, P)
        H9 = mat.project_psd(self._dpk1(F, *self.mp))
        He = self.vol[:, None, None] * np.einsum("nki,nkl,nlj->nij", self.Dfx, H9, self.Dfx)
        return Ee, ge, He

    def barrier_terms(self, x, Y, cand, need_hess=True):
        """kappa * B and its per-pair gradients / projected gel Hessians."""
        total = 0.0
        terms = []
        for kind, (gi, ii) in cand.items():
            if len(gi) == 0:
                continue
            pts = self.pair_points(kind, gi, ii, x, Y)
            gk = "ee" if kind == "ee" else "pt"
            eps = self.eps_x(gi, ii) if kind == "ee" else None
            if not need_hess:
                b = geo.ee_energy_only(pts, self.dhat, eps) if kind == "ee" else geo.pair_barrier(pts, gk, self.dhat, need_hess=False)[0]
                total += self.kappa * float(b.sum())
                continue
            b, g, H = geo.pair_barrier(pts, gk, self.dhat, eps)
            act = b != 0.0
            act |= np.any(g != 0.0, axis=1)
            total += self.kappa * float(b.sum())
            if not np.any(act):
                continue
            gv = self.pair_gel_vertices(kind, gi)[act]
            g, H = self.kappa * g[act], self.kappa * H[act]
            slots = GEL_SLOTS[kind]
            dof = np.concatenate([np.arange(3 * s, 3 * s + 3) for s in slots])
            Hg = mat.project_psd(H[:, dof][:, :, dof])
            terms.append((gv[:, slots], g[:, dof], Hg))
        return total, terms

    def friction_terms(self, x, Y, need_hess=True):
        """Lagged friction potential of the current substep (0 when off)."""
        if self._fric is None:
            return 0.0, []
        pairs, x_t, Y_t = self._fric
        return fric.potential(self, pairs, x, x_t, Y, Y_t, self.mu_f, self.eps_v * self.h, need_hess)

    def energy(self, x, Y, cand, x_tilde=None):
        Ee, _, _ = self.elastic(x, need_hess=False)
        Eb, _ = self.barrier_terms(x, Y, cand, need_hess=False)
        E = Ee + Eb + self.friction_terms(x, Y, need_hess=False)[0]
        if self.dynamic:
            dx = x - x_tilde
            E += 0.5 / (self.h * self.h) * float(np.sum(self.mass[:, None] * dx * dx))
        return E

    def gradient_hessian(self, x, Y, x_tilde=None):
        cand = self.candidates(x, Y)
        Ee, ge, He = self.elastic(x)
        Eb, terms = self.barrier_terms(x, Y, cand)
        Ef, fterms = self.friction_terms(x, Y)
        Eb += Ef
        terms = terms + fterms
        n3 = 3 * self.nv
        g = np.zeros(n3)
        dof = (3 * self.T[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
        np.add.at(g, dof.ravel(), ge.ravel())
        rows = [np.repeat(dof, 12, axis=1).ravel()]
        cols = [np.tile(dof, (1, 12)).ravel()]
        vals = [He.ravel()]
        E = Ee + Eb
        for gv, gg, Hg in terms:
            k = gv.shape[1]
            d = (3 * gv[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 3 * k)
            np.add.at(g, d.ravel(), gg.ravel())
            rows.append(np.repeat(d, 3 * k, axis=1).ravel())
            cols.append(np.tile(d, (1, 3 * k)).ravel())
            vals.append(Hg.ravel())
        if self.dynamic:
            dx = (x - x_tilde).ravel()
            mdiag = np.repeat(self.mass, 3) / (self.h * self.h)
            g += mdiag * dx
            E += 0.5 * float(np.sum(mdiag * dx * dx))
            rows.append(np.arange(n3))
            cols.append(np.arange(n3))
            vals.append(mdiag)
        H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n3, n3)).tocsc()
        return E, g.reshape(-1, 3), H

    # -------------------------------------------------------------- solver
    def ccd_alpha(self, x, p, Y0, Y1=None, t_max=1.0):
        """Largest conservative fraction of the motion (gel x -> x + p,
        indenter Y0 -> Y1) before any pair gets within 10 % of its start
        distance."""
        x1 = x + p
        cand = self.candidates(x, Y0, x1, Y1)
        dY = (Y1 - Y0) if Y1 is not None else np.zeros_like(Y0)
        t = np.inf
        for kind, (gi, ii) in cand.items():
            if len(gi) == 0:
                continue
            pts = self.pair_points(kind, gi, ii, x, Y0)
            disp = self.pair_points(kind, gi, ii, p, dY)
            toi = accd(pts, disp, "ee" if kind == "ee" else "pt", t_max=t_max)
            t = min(t, float(toi.min()))
        return min(t_max, t), cand

    def newton(self, x, Y, x_tilde=None):
        g0 = None
        fr = np.repeat(self.free, 3)
        self.trace.append([])
        for it in range(self.newton_max):
            E, g, H = self.gradient_hessian(x, Y, x_tilde)
            g[~self.free] = 0.0
            gn = float(np.linalg.norm(g))
            if g0 is None:
                g0 = gn
            self.stats["newton"] += 1
            self.trace[-1].append(E)
            if gn <= max(self.rtol * g0, self.gabs):
                return x, it
            Hff = H[fr][:, fr]
            p = np.zeros(3 * self.nv)
            p[fr] = spla.spsolve(Hff.tocsc(), -g.ravel()[fr])
            p = p.reshape(-1, 3)
            alpha, cand = self.ccd_alpha(x, p, Y)
            if np.abs(p).max() <= self.ptol:
                return x + alpha * p, it + 1
            for _ in range(61):
                xt = x + alpha * p
                Et = self.energy(xt, Y, cand, x_tilde)
                if Et <= E:
                    break
                alpha *= 0.5
            else:
                raise LineSearchFail("no decrease after 60 halvings")
            x = xt
        raise NewtonMaxIter(f"no convergence in {self.newton_max} iterations")

    def step(self, target_pose):
        """Advance the indenter to target_pose and solve for the gel."""
        x_t = self.x.copy()
        x_tilde = x_t + self.h * self.v if self.dynamic else None
        Y0 = self.indenter(self.pose)
        Y1 = self.indenter(target_pose)
        x = x_t.copy()
        s = 0.0
        for sub in range(self.max_substeps):
            Ys = (1.0 - s) * Y0 + s * Y1
            if self.friction:  # lagged at the converged state before this substep's advance
                self._fric = (fric.lag(self, x, Ys), x_t, Y0)
            frac, _ = self.ccd_alpha(x, np.zeros_like(x), Ys, Y1)
            s = 1.0 if frac >= 1.0 else s + (1.0 - s) * frac
            Ys = (1.0 - s) * Y0 + s * Y1
            x, _ = self.newton(x, Ys, x_tilde)
            self.stats["substeps"] += 1
            if s >= 1.0:
                break
        else:
            raise NewtonMaxIter("indenter did not reach its target pose")
        if self.dynamic:
            self.v = (x - x_t) / self.h
        self.x = x
        self.pose = target_pose
        self.stats["steps"] += 1
        return x

    # ---------------------------------------------------- stress extraction
    def deformation(self, x=None):
        return msh.deformation_gradient(self.x if x is None else x, self.T, self.Dminv)

    def stress(self, x=None):
        """Eq. 4 per tet, six components (xx, yy, zz, xy, yz, zx)."""
        return mat.sym6(self._cauchy(self.deformation(x), *self.mp))

    def traction(self, x=None, sigma6=None):
        """Algorithm 1 over contact faces: unit outward normal of the deformed
        face, t = sigma n (Eq. 5), p = -n.sigma n (compression positive; the
        paper's p_n of Eq. 7 is -p), t_tau = t - (t.n) n (Eq. 8)."""
        x = self.x if x is None else x
        S = mat.full33(self.stress(x) if sigma6 is None else sigma6)[self.cparent]
        f = self.cfaces
        c = np.cross(x[f[:, 1]] - x[f[:, 0]], x[f[:, 2]] - x[f[:, 0]])
        n = c / np.linalg.norm(c, axis=1, keepdims=True)
        t = np.einsum("nij,nj->ni", S, n)
        pn = np.einsum("ni,ni->n", t, n)
        tt = t - pn[:, None] * n
        return t, -pn, tt

    def vertex_pressure(self, x=None, p_face=None):
        """Area-weighted mean over incident contact faces (deformed areas)."""
        x = self.x if x is None else x
        if p_face is None:
            _, p_face, _ = self.traction(x)
        f = self.cfaces
        A = 0.5 * np.linalg.norm(np.cross(x[f[:, 1]] - x[f[:, 0]], x[f[:, 2]] - x[f[:, 0]]), axis=1)
        out = np.zeros(len(self.cverts))
        for k in range(len(self.cverts)):
            fs = self.csr_idx[self.csr_off[k]:self.csr_off[k + 1]]
            out[k] = np.sum(A[fs] * p_face[fs]) / np.sum(A[fs])
        return out

    def pressure_map(self, x=None, p_vertex=None):
        """Pixel value = barycentric interpolation of the vertex pressure over
        the covering face; uncovered pixels are 0 with mask 0."""
        pv = self.vertex_pressure(x) if p_vertex is None else p_vertex
        slot = -np.ones(self.nv, dtype=np.int64)
        slot[self.cverts] = np.arange(len(self.cverts))
        out = np.zeros(len(self.pix_face))
        cov = self.pix_face >= 0
        f = self.cfaces[self.pix_face[cov]]
        w = self.pix_w[cov].astype(np.float64)
        out[cov] = np.sum(w * pv[slot[f]], axis=1)
        H, W = self.grid["H"], self.grid["W"]
        return out.reshape(H, W), cov.reshape(H, W).astype(np.uint8)

    def contact_force(self, x=None):
        """Total force the indenter exerts on the gel: sum_k f_k with
        f_k = -kappa dB/dx_k (Algorithm 2, f_k = -g_k / dt^2), plus the
        lagged friction force -dD/dx_k of the last substep when friction is
        on."""
        x = self.x if x is None else x
        Y = self.indenter(self.pose)
        _, terms = self.barrier_terms(x, Y, self.candidates(x, Y))
        terms = terms + self.friction_terms(x, Y)[1]
        f = np.zeros(3)
        for gv, gg, _ in terms:
            f -= gg.reshape(len(gv), -1, 3).sum(axis=(0, 1))
        return f

    def vertex_contact_forces(self, x=None):
        """Algorithm 2's contact decomposition at every contact-surface vertex
        k (sorted ids, as self.cverts): the contact force f_k = -g_k of the
        barrier (and friction) part of the potential (the potential is divided
        by dt^2, so this is Algorithm 2's -g_k / dt^2), the unit vertex normal
        n_k (the area-weighted mean of the incident deformed contact faces'
        outward normals), the vertex area A_k (a third of each incident face's
        deformed area), f_n = (f.n) n, f_tau = f - f_n and p_k = |f_k| / A_k.
        Returns (f, f_n, f_tau, p, n, A)."""
        x = self.x if x is None else x
        Y = self.indenter(self.pose)
        _, terms = self.barrier_terms(x, Y, self.candidates(x, Y))
        terms = terms + self.friction_terms(x, Y)[1]
        g = np.zeros((self.nv, 3))
        for gv, gg, _ in terms:
            np.add.at(g, gv.ravel(), gg.reshape(-1, 3))
        f = -g[self.cverts]
        nk, Ak = self.vertex_normals_areas(x)
        fn = np.einsum("ki,ki->k", f, nk)[:, None] * nk
        return f, fn, f - fn, np.linalg.norm(f, axis=1) / Ak, nk, Ak

    def vertex_normals_areas(self, x=None):
        """Per contact-surface vertex: the unit normal (area-weighted mean of
        the incident deformed contact faces' outward normals) and the area (a
        third of the incident faces' deformed areas)."""
        x = self.x if x is None else x
        fc = self.cfaces
        c = np.cross(x[fc[:, 1]] - x[fc[:, 0]], x[fc[:, 2]] - x[fc[:, 0]])   # 2 A_f n_f
        nk = np.zeros((len(self.cverts), 3))
        Ak = np.zeros(len(self.cverts))
        for k in range(len(self.cverts)):
            fs = self.csr_idx[self.csr_off[k]:self.csr_off[k + 1]]
            s = c[fs].sum(axis=0)
            nk[k] = s / np.linalg.norm(s)
            Ak[k] = np.sum(0.5 * np.linalg.norm(c[fs], axis=1)) / 3.0
        return nk, Ak

    def force_pressure_map(self, x=None):
        """The contact-force pressure p_k = |f_k| / A_k of Algorithm 2 on the
        pixel grid (the same barycentric splat as the stress-based map)."""
        p = self.vertex_contact_forces(x)[3]
        return self.pressure_map(p_vertex=p)

    def depth_map(self, x=None, grid=None):
        """Height of the deformed contact surface seen from the contact side,
        on the pixel grid: every deformed contact face is projected on the
        grid plane ((axis_u, axis_v) coordinates); at each pixel centre
        covered by a projected face (closed triangle, either orientation) the
        face's outward height (the thickness-axis coordinate times the
        outward sign) is interpolated barycentrically; the map holds the
        largest such height over the covering faces, rounded to FP32 (the
        surface nearest the indenter, a z-buffer), and 0 with mask 0 where no
        face covers the centre.  The first stage of the optical rendering of
        Sec. III-D (the depth the renderer is constrained to)."""
        x = self.x if x is None else x
        g = self.grid if grid is None else grid
        au, av, H, W = g["axis_u"], g["axis_v"], g["H"], g["W"]
        pu = g["origin"][0] + (np.arange(W) + 0.5) * g["pixel"][0]
        pv = g["origin"][1] + (np.arange(H) + 0.5) * g["pixel"][1]
        best = np.full(H * W, -np.inf, dtype=np.float32)
        U, V = x[:, au], x[:, av]
        h = self.out_sign * x[:, self.thick_axis]
        for a, b, c in self.cfaces:
            A2 = (U[b] - U[a]) * (V[c] - V[a]) - (V[b] - V[a]) * (U[c] - U[a])
            if A2 == 0:
                continue
            cs = np.nonzero((pu >= min(U[a], U[b], U[c])) & (pu <= max(U[a], U[b], U[c])))[0]
            rs = np.nonzero((pv >= min(V[a], V[b], V[c])) & (pv <= max(V[a], V[b], V[c])))[0]
            if len(cs) == 0 or len(rs) == 0:
                continue
            PU, PV = np.meshgrid(pu[cs], pv[rs])
            ea = (U[c] - U[b]) * (PV - V[b]) - (V[c] - V[b]) * (PU - U[b])
            eb = (U[a] - U[c]) * (PV - V[c]) - (V[a] - V[c]) * (PU - U[c])
            ec = (U[b] - U[a]) * (PV - V[a]) - (V[b] - V[a]) * (PU - U[a])
            inside = ((ea >= 0) & (eb >= 0) & (ec >= 0)) | ((ea <= 0) & (eb <= 0) & (ec <= 0))
            R, C = np.meshgrid(rs, cs, indexing="ij")
            pix = (R * W + C)[inside]
            val = ((ea[inside] * h[a] + eb[inside] * h[b] + ec[inside] * h[c]) / A2).astype(np.float32)
            np.maximum.at(best, pix, val)
        mask = np.isfinite(best)
        out = np.where(mask, best, np.float32(0.0)).astype(np.float32)
        return out.reshape(H, W), mask.reshape(H, W).astype(np.uint8)

    def reaction_force(self, x=None):
        """Sum over fixed vertices of the elastic force the gel exerts on its
        support (equals the contact force at quasi-static equilibrium)."""
        x = self.x if x is None else x
        _, ge, _ = self.elastic(x)
        g = np.zeros((self.nv, 3))
        np.add.at(g, self.T.ravel(), ge.reshape(-1, 3))
        return g[self.fixed].sum(axis=0)


def _segment_hits_triangle(E, F):
    """Closed segment E (n,2,3) meets triangle F (n,3,3) (exact sign tests in
    FP64; touching counts as a hit)."""
    a, b = E[:, 0], E[:, 1]
    p0, p1, p2 = F[:, 0], F[:, 1], F[:, 2]

    def orient(q0, q1, q2, q3):
        return np.einsum("ni,ni->n", q1 - q0, np.cross(q2 - q0, q3 - q0))
    sa = orient(p0, p1, p2, a)
    sb = orient(p0, p1, p2, b)
    straddle = ((sa <= 0) & (sb >= 0)) | ((sa >= 0) & (sb <= 0))
    s0 = orient(a, b, p0, p1)
    s1 = orient(a, b, p1, p2)
    s2 = orient(a, b, p2, p0)
    inside = ((s0 >= 0) & (s1 >= 0) & (s2 >= 0)) | ((s0 <= 0) & (s1 <= 0) & (s2 <= 0))
    coplanar = (sa == 0) & (sb == 0)
    return straddle & inside & ~coplanar
