"""Mesh-side setup (oracle, FP64 / exact integers).

* rest shape: Dm = [X1-X0, X2-X0, X3-X0], V = det(Dm)/6 (tets with det <= 0
  are rejected), F = Ds Dm^-1.
* Algorithm 1, first three steps: surface triangles with their parent tets.
  The four faces of tet (0,1,2,3) are taken as (1,2,3), (0,3,2), (0,1,3),
  (0,2,1), which are outward for a positively oriented tet.  A face is on the
  boundary iff its vertex set occurs once; faces are ordered by their sorted
  vertex triple; the stored triple is the outward winding rotated so that
  its smallest vertex id comes first.
* contact band (Sec. III-A): the thickness axis is the thinnest bounding-box
  axis; vertices within 15 % of the thickness of the face opposite the fixed
  side form the band; contact faces are boundary faces with all three vertices
  in the band.
* vertex/face incidence over contact faces for area-weighted averaging.
* pixel binning: rest coordinates snapped to integer nanometres, exact
  integer edge functions, lowest covering face wins, FP64 barycentrics.
"""
import numpy as np

TET_FACES = np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])


class InvalidMesh(ValueError):
    pass


def rest_shape(X, T):
    """Dm^-1 (nt,3,3) and rest volume (nt,)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T)
    Dm = np.stack([X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]],
                   X[T[:, 3]] - X[T[:, 0]]], axis=2)
    det = np.linalg.det(Dm)
    if np.any(~(det > 0.0)):
        raise InvalidMesh(f"{int(np.sum(~(det > 0)))} tets with non-positive orientation")
    return np.linalg.inv(Dm), det / 6.0


def deformation_gradient(x, T, Dminv):
    Ds = np.stack([x[T[:, 1]] - x[T[:, 0]], x[T[:, 2]] - x[T[:, 0]],
                   x[T[:, 3]] - x[T[:, 0]]], axis=2)
    return Ds @ Dminv


def dF_dx(Dminv):
    """(nt, 9, 12) Jacobian of vec(F) (row-major) w.r.t. the 12 vertex
    coordinates (vertex-major, xyz-minor): dF_ij/dx_{a,k} = delta_ik n_a[j]
    with n_a = row (a-1) of Dm^-1 for a >= 1 and n_0 = -(n_1+n_2+n_3)."""
    nt = Dminv.shape[0]
    n = np.empty((nt, 4, 3))
    n[:, 1:, :] = Dminv
    n[:, 0, :] = -Dminv.sum(axis=1)
    D = np.zeros((nt, 3, 3, 4, 3))
    for i in range(3):
        D[:, i, :, :, i] = np.swapaxes(n, 1, 2)
    return D.reshape(nt, 9, 12)


def lumped_mass(T, vol, density, nv):
    m = np.zeros(nv)
    np.add.at(m, T.ravel(), np.repeat(density * vol / 4.0, 4))
    return m


def boundary_faces(T):
    """Boundary triangles (nf,3) with outward winding and their parent tet
    (nf,), in lexicographic order of the sorted vertex triple."""
    T = np.asarray(T)
    nt = T.shape[0]
    faces = T[:, TET_FACES].reshape(-1, 3)
    parent = np.repeat(np.arange(nt), 4)
    key = np.sort(faces, axis=1)
    uniq, inv, counts = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    once = counts[inv.ravel()] == 1
    faces, parent, key = faces[once], parent[once], key[once]
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    faces, parent = faces[order], parent[order]
    # rotate each triple so that its smallest id comes first (winding kept)
    r = np.argmin(faces, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    faces = np.take_along_axis(faces, idx, axis=1)
    return faces.astype(np.int32), parent.astype(np.int32)


def thickness_axis(X, axis=-1):
    if axis >= 0:
        return int(axis)
    ext = X.max(axis=0) - X.min(axis=0)
    return int(np.argmin(ext))  # first minimal axis on ties


def contact_band(X, fixed, axis=-1, frac=0.15):
    """Boolean band mask: vertices within frac * thickness of the side
    opposite the fixed set (top side when nothing is fixed)."""
    a = thickness_axis(X, axis)
    c = X[:, a]
    lo, hi = c.min(), c.max()
    thick = hi - lo
    top = True
    if len(fixed) > 0:
        top = X[np.asarray(fixed), a].mean() <= 0.5 * (lo + hi)
    if top:
        return c >= hi - frac * thick
    return c <= lo + frac * thick


def contact_faces(faces, band):
    sel = np.nonzero(band[faces].all(axis=1))[0]
    return sel.astype(np.int32)


def surface_edges(faces):
    """Unique undirected edges (a < b) of a triangle set, lexicographic."""
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0).astype(np.int32)


def vertex_face_csr(faces):
    """Sorted unique vertices of ``faces`` and, per vertex, the indices of
    the incident faces in increasing order (CSR offsets, indices)."""
    verts = np.unique(faces.ravel())
    pairs = np.stack([faces.ravel(), np.repeat(np.arange(len(faces)), 3)], axis=1)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    pairs = pairs[order]
    counts = np.searchsorted(pairs[:, 0], verts, side="right") - np.searchsorted(pairs[:, 0], verts, side="left")
    off = np.concatenate([[0], np.cumsum(counts)])
    return verts.astype(np.int32), off.astype(np.int32), pairs[:, 1].astype(np.int32)


# ---------------------------------------------------------------- pixel binning

def snap_nm(x):
    """Round metres to integer nanometres (round half to even)."""
    return np.rint(np.asarray(x, dtype=np.float64) * 1e9).astype(np.int64)


def _edge(au, av, bu, bv, pu, pv):
    return (bu - au) * (pv - av) - (bv - av) * (pu - au)


def bin_pixels(X, faces, grid):
    """Covering face and barycentric weights for every pixel of ``grid``.

    Pixel (r, c) has centre (u0 + (c+1/2) du, v0 + (r+1/2) dv) in the
    (axis_u, axis_v) plane of the rest configuration.  All coordinates are
    snapped to nanometres and doubled, so that centres are integers and the
    edge functions are exact int64.  A face covers a pixel if the three edge
    functions have the sign of its doubled area (zero allowed); the lowest
    face index wins.  Returns pix_face (H*W,) int32 (-1 = uncovered) and
    pix_w (H*W, 3) float32 = (E_bc, E_ca, E_ab) / A in FP64, rounded once.
    """
    au, av = grid["axis_u"], grid["axis_v"]
    H, W = grid["H"], grid["W"]
    U = 2 * snap_nm(X[:, au])
    Vv = 2 * snap_nm(X[:, av])
    u0, v0 = snap_nm(grid["origin"][0]), snap_nm(grid["origin"][1])
    du, dv = snap_nm(grid["pixel"][0]), snap_nm(grid["pixel"][1])
    pu = 2 * u0 + (2 * np.arange(W, dtype=np.int64) + 1) * du   # doubled centres
    pv = 2 * v0 + (2 * np.arange(H, dtype=np.int64) + 1) * dv
    pix_face = np.full(H * W, -1, dtype=np.int64)
    pix_w = np.zeros((H * W, 3), dtype=np.float32)
    best = np.full(H * W, np.iinfo(np.int64).max, dtype=np.int64)
    for f in range(len(faces)):
        a, b, c = faces[f]
        A2 = _edge(U[a], Vv[a], U[b], Vv[b], U[c], Vv[c])
        if A2 == 0:
            continue
        umin, umax = min(U[a], U[b], U[c]), max(U[a], U[b], U[c])
        vmin, vmax = min(Vv[a], Vv[b], Vv[c]), max(Vv[a], Vv[b], Vv[c])
        cs = np.nonzero((pu >= umin) & (pu <= umax))[0]
        rs = np.nonzero((pv >= vmin) & (pv <= vmax))[0]
        if len(cs) == 0 or len(rs) == 0:
            continue
        PU, PV = np.meshgrid(pu[cs], pv[rs])
        ea = _edge(U[b], Vv[b], U[c], Vv[c], PU, PV)
        eb = _edge(U[c], Vv[c], U[a], Vv[a], PU, PV)
        ec = _edge(U[a], Vv[a], U[b], Vv[b], PU, PV)
        if A2 > 0:
            inside = (ea >= 0) & (eb >= 0) & (ec >= 0)
        else:
            inside = (ea <= 0) & (eb <= 0) & (ec <= 0)
        R, C = np.meshgrid(rs, cs, indexing="ij")
        pix = (R * W + C)[inside]
        take = f < best[pix]
        pix = pix[take]
        best[pix] = f
        pix_face[pix] = f
        A2f = np.float64(A2)
        pix_w[pix, 0] = (ea[inside][take].astype(np.float64) / A2f).astype(np.float32)
        pix_w[pix, 1] = (eb[inside][take].astype(np.float64) / A2f).astype(np.float32)
        pix_w[pix, 2] = (ec[inside][take].astype(np.float64) / A2f).astype(np.float32)
    return pix_face.astype(np.int32), pix_w
