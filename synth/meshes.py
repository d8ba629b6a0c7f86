"""Structured tetrahedral gel meshes (inputs only).

Every mesh is a tensor-product hexahedral grid, possibly mapped, split into six
tetrahedra per hex along the cube's main diagonal (the Kuhn / Freudenthal
split).  Vertex ids are ``i + (nx+1)*(j + (ny+1)*k)``; tets are positively
oriented (det[x1-x0, x2-x0, x3-x0] > 0).

Shapes (stand-ins for the sensors of Sec. IV; the paper meshes real sensor
CAD with WildMeshing, which is not available here):
  * ``box``          - uniform box (the 1,800-tet 20x20x4 mm pad).
  * ``graded_pad``   - GelSight-Mini-like pad refined toward the contact face
                       with the radial profile of Sec. III-A (fine core at 40 %
                       of the half-extent, cosine transition over 20 %).
  * ``dome``         - DIGIT-like spherical cap on a base slab.
  * ``block``        - 9DTact-like block.
"""
import numpy as np

# Path order of the six Kuhn tets: permutations of the axes (x=0, y=1, z=2).
_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_ODD = {(0, 2, 1), (1, 0, 2), (2, 1, 0)}


def kuhn_grid(xs, ys, zs, zmap=None):
    """Split the tensor grid xs x ys x zs into 6 tets per hex.

    zmap(x, y, z) -> z' optionally remaps heights (used by the dome).
    Returns X (nv, 3) float64 and tets (nt, 4) int32.
    """
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (xs, ys, zs))
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    X = np.stack([xs[I.ravel()], ys[J.ravel()], zs[K.ravel()]], axis=1)
    if zmap is not None:
        X[:, 2] = zmap(X[:, 0], X[:, 1], X[:, 2])

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    tets = []
    for perm in _KUHN_PERMS:
        c = [np.zeros_like(i), np.zeros_like(i), np.zeros_like(i)]
        path = [vid(i, j, k)]
        for ax in perm:
            c[ax] = c[ax] + 1
            path.append(vid(i + c[0], j + c[1], k + c[2]))
        if perm in _ODD:
            path[1], path[2] = path[2], path[1]
        tets.append(np.stack(path, axis=1))
    # interleave so the six tets of one hex are adjacent in memory
    T = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return X, T


def box(nx, ny, nz, Lx, Ly, Lz):
    """Uniform box [0,Lx]x[0,Ly]x[0,Lz] (metres)."""
    return kuhn_grid(np.linspace(0, Lx, nx + 1), np.linspace(0, Ly, ny + 1),
                     np.linspace(0, Lz, nz + 1))


def _graded_nodes(length, h_of, scale, center=True):
    """Node coordinates on [0, length] whose local spacing follows scale*h_of(x).

    The cumulative cell count u(x) = int dx / h(x) is tabulated and inverted,
    so that nodes are u^-1(i * u(L) / N) with N = round(u(L) / scale).
    """
    t = np.linspace(0.0, length, 40001)
    inv = 1.0 / h_of(t)
    u = np.concatenate([[0.0], np.cumsum(0.5 * (inv[1:] + inv[:-1]) * np.diff(t))])
    n = max(1, int(round(u[-1] / scale)))
    nodes = np.interp(np.linspace(0.0, u[-1], n + 1), u, t)
    nodes[0], nodes[-1] = 0.0, length
    if center:  # enforce mirror symmetry about the midpoint
        nodes = 0.5 * (nodes + (length - nodes[::-1]))
    return nodes


def _radial_profile(half, h_fine, h_coarse, r_core=0.4, r_band=0.2):
    """Spacing vs. offset from the centre: fine inside r_core*half, cosine
    blend over r_band*half, coarse outside (the profile of Sec. III-A)."""
    rc, rt = r_core * half, r_band * half

    def h(x):
        r = np.abs(x - half)
        s = np.clip((r - rc) / rt, 0.0, 1.0)
        return h_fine + (h_coarse - h_fine) * 0.5 * (1.0 - np.cos(np.pi * s))
    return h


def graded_pad(Lx=18e-3, Ly=24e-3, Lz=4e-3, h_fine=0.25e-3, h_coarse=1e-3,
               target_tets=60000, tol=0.10):
    """GelSight-Mini-like pad: x/y spacing h_fine in the core, h_coarse at the
    rim; z spacing h_fine at the top (contact face, z=Lz) to h_coarse at the
    bottom.  All spacings are scaled by one factor so that the tet count is
    within +-tol of target_tets."""
    hx = _radial_profile(Lx / 2, h_fine, h_coarse)
    hy = _radial_profile(Ly / 2, h_fine, h_coarse)

    def hz(z):
        return h_coarse + (h_fine - h_coarse) * (z / Lz)

    def build(scale):
        xs = _graded_nodes(Lx, hx, scale)
        ys = _graded_nodes(Ly, hy, scale)
        zs = _graded_nodes(Lz, hz, scale, center=False)
        return xs, ys, zs

    lo, hi = 0.2, 5.0
    best = None
    for _ in range(60):
        mid = np.sqrt(lo * hi)
        xs, ys, zs = build(mid)
        nt = 6 * (len(xs) - 1) * (len(ys) - 1) * (len(zs) - 1)
        if best is None or abs(nt - target_tets) < abs(best[0] - target_tets):
            best = (nt, xs, ys, zs)
        if abs(nt - target_tets) <= tol * target_tets:
            break
        if nt > target_tets:
            lo = mid
        else:
            hi = mid
    _, xs, ys, zs = best
    return kuhn_grid(xs, ys, zs)


def dome(Lx=20e-3, Ly=16e-3, cap_radius=30e-3, cap_height=3e-3, slab=1.5e-3,
         nx=24, ny=20, nz=8):
    """DIGIT-like dome: a spherical cap (radius cap_radius, apex height
    cap_height above the slab) clipped to the Lx x Ly base, on a base slab of
    thickness ``slab``.  The column above (x, y) is split uniformly in z."""
    xs = np.linspace(0, Lx, nx + 1)
    ys = np.linspace(0, Ly, ny + 1)
    zs = np.linspace(0, 1.0, nz + 1)
    zc = slab + cap_height - cap_radius

    def top(x, y):
        r2 = (x - Lx / 2) ** 2 + (y - Ly / 2) ** 2
        return np.maximum(slab, zc + np.sqrt(np.maximum(cap_radius ** 2 - r2, 0.0)))

    return kuhn_grid(xs, ys, zs, zmap=lambda x, y, z: z * top(x, y))


def block(nx=30, ny=30, nz=5, Lx=30e-3, Ly=30e-3, Lz=5e-3):
    """9DTact-like block."""
    return box(nx, ny, nz, Lx, Ly, Lz)


def hertz_block(L=20e-3, H=10e-3, h_fine=0.12e-3, h_coarse=1.5e-3, r_core=1.8e-3, r_band=3.0e-3):
    """Block [0,L]^2 x [0,H] for the sphere-indentation check: x/y spacing
    h_fine within r_core of the centre, blending (cosine) to h_coarse over
    r_band; z spacing h_fine at the top, growing linearly towards h_coarse at
    the bottom."""
    def hxy(x):
        r = np.abs(x - L / 2)
        s = np.clip((r - r_core) / r_band, 0.0, 1.0)
        return h_fine + (h_coarse - h_fine) * 0.5 * (1.0 - np.cos(np.pi * s))

    def hz(z):
        d = H - z
        return np.minimum(h_coarse, h_fine + 0.35 * d)

    xs = _graded_nodes(L, hxy, 1.0)
    zs = _graded_nodes(H, hz, 1.0, center=False)
    return kuhn_grid(xs, xs, zs)

