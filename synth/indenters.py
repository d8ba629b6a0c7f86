"""Rigid indenter surface meshes in their body frame (inputs only).

Each function returns V (n, 3) float64 metres and F (m, 3) int32 with
outward-facing counter-clockwise triangles.  The body frame puts the shape's
lowest point at z = -half_height so that a pose translation t places it at
t_z - half_height; ``lowest_z`` returns that offset.
"""
import numpy as np


def icosphere(radius, level):
    """Sphere by ``level`` rounds of 4:1 subdivision of an icosahedron,
    midpoints pushed onto the sphere.  Edge length ~ 1.05 * radius / 2**level."""
    p = (1.0 + 5 ** 0.5) / 2.0
    V = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p),
         (0, -1, -p), (0, 1, -p), (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    for _ in range(level):
        cache = {}
        newF = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = newF
    return np.array(V) * radius, np.array(F, dtype=np.int32)


def cylinder(radius, length, h):
    """Capped cylinder along the body x axis, centred at the origin, with
    surface edge length about h (rings every h, ~2*pi*R/h segments)."""
    nseg = max(8, int(np.ceil(2 * np.pi * radius / h)))
    nring = max(1, int(np.ceil(length / h)))
    xs = np.linspace(-length / 2, length / 2, nring + 1)
    th = 2 * np.pi * np.arange(nseg) / nseg
    V = [np.array([x, radius * np.cos(t), radius * np.sin(t)]) for x in xs for t in th]
    F = []
    for r in range(nring):
        for s in range(nseg):
            a = r * nseg + s
            b = r * nseg + (s + 1) % nseg
            c = (r + 1) * nseg + s
            d = (r + 1) * nseg + (s + 1) % nseg
            F += [(a, b, d), (a, d, c)]
    # end caps: concentric rings down to a centre vertex
    ncap = max(1, int(np.ceil(radius / h)))
    for side, x in ((0, xs[0]), (1, xs[-1])):
        outer = [(0 if side == 0 else nring) * nseg + s for s in range(nseg)]
        for k in range(ncap - 1, 0, -1):
            rr = radius * k / ncap
            inner = []
            for t in th:
                V.append(np.array([x, rr * np.cos(t), rr * np.sin(t)]))
                inner.append(len(V) - 1)
            for s in range(nseg):
                a, b = outer[s], outer[(s + 1) % nseg]
                c, d = inner[s], inner[(s + 1) % nseg]
                if side == 0:
                    F += [(a, c, d), (a, d, b)]
                else:
                    F += [(a, b, d), (a, d, c)]
            outer = inner
        V.append(np.array([x, 0.0, 0.0]))
        ctr = len(V) - 1
        for s in range(nseg):
            a, b = outer[s], outer[(s + 1) % nseg]
            F.append((a, ctr, b) if side == 0 else (a, b, ctr))
    return np.array(V), np.array(F, dtype=np.int32)


def rounded_box(half, fillet, h):
    """Box of half-extents ``half`` (3,) whose edges and corners are rounded
    with radius ``fillet``: each face of the bounding cube is gridded at
    spacing ~h and every grid point q is mapped to c + fillet*(q-c)/|q-c|,
    c = q clamped to the inner box (half - fillet)."""
    half = np.asarray(half, dtype=np.float64)
    inner = half - fillet
    V, F = [], []
    index = {}

    def vert(q):
        key = tuple(np.round(q / (h * 1e-3)).astype(np.int64))
        if key in index:
            return index[key]
        c = np.clip(q, -inner, inner)
        d = q - c
        n = np.linalg.norm(d)
        p = c + fillet * d / n if n > 0 else q
        V.append(p)
        index[key] = len(V) - 1
        return index[key]

    for ax in range(3):
        u, v = (ax + 1) % 3, (ax + 2) % 3
        nu = max(2, int(np.ceil(2 * half[u] / h)))
        nv = max(2, int(np.ceil(2 * half[v] / h)))
        us = np.linspace(-half[u], half[u], nu + 1)
        vs = np.linspace(-half[v], half[v], nv + 1)
        for sgn in (-1.0, 1.0):
            ids = np.empty((nu + 1, nv + 1), dtype=np.int64)
            for a in range(nu + 1):
                for b in range(nv + 1):
                    q = np.zeros(3)
                    q[ax], q[u], q[v] = sgn * half[ax], us[a], vs[b]
                    ids[a, b] = vert(q)
            for a in range(nu):
                for b in range(nv):
                    p00, p10, p01, p11 = ids[a, b], ids[a + 1, b], ids[a, b + 1], ids[a + 1, b + 1]
                    if sgn > 0:
                        F += [(p00, p10, p11), (p00, p11, p01)]
                    else:
                        F += [(p00, p11, p10), (p00, p01, p11)]
    return np.array(V), np.array(F, dtype=np.int32)


def lowest_z(V):
    """Offset from the body origin to the lowest vertex (negative)."""
    return float(V[:, 2].min())
