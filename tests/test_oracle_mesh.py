"""Pins for oracle/mesh.py: boundary extraction against a brute-force face
count and the divergence theorem, contact band on the 1,800-tet pad, rest
volumes, the F(x) Jacobian, and pixel binning against exact Python-integer
brute force and linear-field reproduction."""
import numpy as np
import pytest

from oracle import mesh as msh
from synth import meshes, workloads


@pytest.fixture(scope="module")
def pad():
    X, T = meshes.box(10, 10, 3, 20e-3, 20e-3, 4e-3)
    return X, T


def test_rest_volume_and_orientation(pad):
    X, T = pad
    Dminv, vol = msh.rest_shape(X, T)
    assert np.all(vol > 0)
    assert vol.sum() == pytest.approx(20e-3 * 20e-3 * 4e-3, rel=1e-12)
    bad = T.copy()
    bad[0, [1, 2]] = bad[0, [2, 1]]
    with pytest.raises(msh.InvalidMesh):
        msh.rest_shape(X, bad)


def test_boundary_faces_bruteforce(pad):
    X, T = pad
    faces, parent = msh.boundary_faces(T)
    # brute force: count every tet face by its vertex set with a dict
    count = {}
    for t in T:
        for f in msh.TET_FACES:
            k = tuple(sorted(t[f]))
            count[k] = count.get(k, 0) + 1
    once = sorted(k for k, c in count.items() if c == 1)
    assert len(faces) == len(once) == 2 * (10 * 10 * 2) + 2 * (2 * 10 * 3 * 2)  # 640
    assert [tuple(sorted(f)) for f in faces] == once           # canonical order
    assert np.all(faces[:, 0] == faces.min(axis=1))            # min id first
    for f, p in zip(faces, parent):
        assert set(f) <= set(T[p])
    # every boundary face lies on a face of the box
    lo, hi = X.min(axis=0), X.max(axis=0)
    P = X[faces]
    on = np.zeros(len(faces), dtype=bool)
    for a in range(3):
        on |= np.all(P[:, :, a] == lo[a], axis=1) | np.all(P[:, :, a] == hi[a], axis=1)
    assert on.all()


def test_boundary_winding_is_outward(pad):
    """Divergence theorem on the closed surface: sum n_f A_f = 0 and
    sum (c_f . n_f) A_f = 3 V, which fails if any face is wound inward."""
    X, T = pad
    faces, _ = msh.boundary_faces(T)
    P = X[faces]
    an = 0.5 * np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    assert np.abs(an.sum(axis=0)).max() < 1e-15
    c = P.mean(axis=1)
    assert np.einsum("ij,ij->", c, an) == pytest.approx(3 * 20e-3 * 20e-3 * 4e-3, rel=1e-12)
    # each face points away from its parent's fourth vertex
    _, parent = msh.boundary_faces(T)
    for f, p in zip(faces[:50], parent[:50]):
        other = [v for v in T[p] if v not in f][0]
        n = np.cross(X[f[1]] - X[f[0]], X[f[2]] - X[f[0]])
        assert np.dot(X[other] - X[f[0]], n) < 0


def test_contact_band_is_top_face(pad):
    X, T = pad
    fixed = np.nonzero(X[:, 2] == 0)[0]
    faces, _ = msh.boundary_faces(T)
    band = msh.contact_band(X, fixed)
    cf = msh.contact_faces(faces, band)
    assert len(cf) == 200
    assert np.all(X[faces[cf]][:, :, 2] == 4e-3)
    assert msh.thickness_axis(X) == 2
    # fixed on top -> band at the bottom
    band2 = msh.contact_band(X, np.nonzero(X[:, 2] == 4e-3)[0])
    assert np.all(X[band2, 2] == 0.0)
    e = msh.surface_edges(faces[cf])
    assert len(e) == 2 * 10 * 11 + 100  # grid edges + one diagonal per cell
    verts, off, idx = msh.vertex_face_csr(faces[cf])
    assert len(verts) == 121 and off[-1] == 600
    for k, v in enumerate(verts):
        fs = idx[off[k]:off[k + 1]]
        assert np.all(np.diff(fs) > 0)
        assert all(v in faces[cf][f] for f in fs)


def test_dF_dx_is_the_jacobian(pad):
    X, T = pad
    Dminv, _ = msh.rest_shape(X, T)
    D = msh.dF_dx(Dminv)
    rng = np.random.default_rng(0)
    x = X + 1e-4 * rng.standard_normal(X.shape)
    F = msh.deformation_gradient(x, T, Dminv)
    u = (x - X)[T].reshape(-1, 12)
    assert np.allclose(F.reshape(-1, 9), np.eye(3).ravel() + np.einsum("nij,nj->ni", D, u), atol=1e-12)


def test_lumped_mass_total(pad):
    X, T = pad
    _, vol = msh.rest_shape(X, T)
    m = msh.lumped_mass(T, vol, 1100.0, len(X))
    assert m.sum() == pytest.approx(1100.0 * vol.sum(), rel=1e-12)


def _bruteforce_bins(X, faces, grid):
    """Pure-Python integers, every pixel against every face."""
    au, av = grid["axis_u"], grid["axis_v"]
    q = lambda v: int(round(v * 1e9)) if abs(v * 1e9 - round(v * 1e9)) != 0.5 else int(np.rint(v * 1e9))
    U = [2 * q(x) for x in X[:, au]]
    V = [2 * q(x) for x in X[:, av]]
    u0, v0 = q(grid["origin"][0]), q(grid["origin"][1])
    du, dv = q(grid["pixel"][0]), q(grid["pixel"][1])
    out = []
    for r in range(grid["H"]):
        for c in range(grid["W"]):
            pu, pv = 2 * u0 + (2 * c + 1) * du, 2 * v0 + (2 * r + 1) * dv
            hit = -1
            for fi, (a, b, cc) in enumerate(faces):
                def cross(i, j):
                    return (U[j] - U[i]) * (pv - V[i]) - (V[j] - V[i]) * (pu - U[i])
                A = (U[b] - U[a]) * (V[cc] - V[a]) - (V[b] - V[a]) * (U[cc] - U[a])
                e = (cross(b, cc), cross(cc, a), cross(a, b))
                if A != 0 and (all(x >= 0 for x in e) if A > 0 else all(x <= 0 for x in e)):
                    hit = fi
                    break
            out.append(hit)
    return np.array(out)


def test_binning_matches_bruteforce_and_reproduces_linear_fields():
    env = workloads.pad_env(0, nx=4, ny=4, nz=2, size=(8e-3, 8e-3, 2e-3), grid_hw=(12, 12))
    X, T, grid = env["X"], env["tets"], env["grid"]
    faces, _ = msh.boundary_faces(T)
    cf = faces[msh.contact_faces(faces, msh.contact_band(X, env["fixed"]))]
    pf, pw = msh.bin_pixels(X, cf, grid)
    assert np.array_equal(pf, _bruteforce_bins(X, cf, grid))
    # many pixel centres sit exactly on cell diagonals -> ties resolved low
    assert np.all(pf >= 0)
    # barycentric weights reproduce the pixel centre (a linear field); the
    # grid is snapped to whole nanometres (0.67 mm pixels: < 0.5 nm per step)
    r, c = np.divmod(np.arange(grid["H"] * grid["W"]), grid["W"])
    cu = grid["origin"][0] + (c + 0.5) * grid["pixel"][0]
    cv = grid["origin"][1] + (r + 0.5) * grid["pixel"][1]
    P = X[cf[pf]]
    w = pw.astype(np.float64)
    assert np.abs(np.sum(w * P[:, :, 0], axis=1) - cu).max() < 1e-8
    assert np.abs(np.sum(w * P[:, :, 1], axis=1) - cv).max() < 1e-8
    assert np.abs(w.sum(axis=1) - 1).max() < 1e-6


def test_binning_uncovered_pixels():
    X, T = meshes.box(2, 2, 1, 4e-3, 4e-3, 1e-3)
    faces, _ = msh.boundary_faces(T)
    cf = faces[msh.contact_faces(faces, msh.contact_band(X, np.nonzero(X[:, 2] == 0)[0]))]
    grid = dict(axis_u=0, axis_v=1, origin=(-1e-3, -1e-3), pixel=(0.5e-3, 0.5e-3), H=12, W=12)
    pf, pw = msh.bin_pixels(X, cf, grid)
    assert np.array_equal(pf, _bruteforce_bins(X, cf, grid))
    r, c = np.divmod(np.arange(144), 12)
    cu = -1e-3 + (c + 0.5) * 0.5e-3
    cv = -1e-3 + (r + 0.5) * 0.5e-3
    inside = (cu > 0) & (cu < 4e-3) & (cv > 0) & (cv < 4e-3)
    assert np.array_equal(pf >= 0, inside)
    assert np.all(pw[pf < 0] == 0)
