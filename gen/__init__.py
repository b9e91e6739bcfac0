"""Seeded synthetic inputs: triangle meshes and query points.

This module holds input generation only.  It contains none of the winding-number
arithmetic (no solid angles, no predicates, no boundary extraction); both the
CUDA library and the CPU oracle consume what it produces.

Every array it returns is a plain numpy array:

* vertices ``V``: ``float32[nv, 3]``
* faces ``F``: ``int32[nt, 3]`` (counter-clockwise seen from outside)
* queries ``Q``: ``float32[n, 3]``

Randomness always comes from ``numpy.random.default_rng(seed)`` (PCG64), one
stream per workload, consumed in the order each function documents.  The
workloads mirror the shapes the paper evaluates on (Sec. 5): open meshes with
boundary (holes), self-intersecting soups, closed meshes, and a robustness test
with exactly-representable degenerate queries (Supp. S2, robustness figure).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "icosahedron", "subdivide", "icosphere", "small_cap", "displaced_soup",
    "queries_uniform_bbox", "queries_near_surface", "staircase_sphere",
    "height_field_patch", "precision_workload", "grid_queries", "superquadric",
    "random_soup", "batched_workload", "workload", "bezier_patches", "param_workload",
]


@dataclass
class Mesh:
    V: np.ndarray                     # float32 [nv, 3]
    F: np.ndarray                     # int32   [nt, 3]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.V.shape[0])

    @property
    def nt(self) -> int:
        return int(self.F.shape[0])


# ----------------------------------------------------------------------------
# Icosphere
# ----------------------------------------------------------------------------

def icosahedron():
    """Regular icosahedron on the unit sphere, faces oriented outward.

    Vertices are the 12 cyclic permutations of (0, +-1, +-phi), normalised.
    Faces are found as the 20 triples of mutually adjacent vertices (edge length
    2 before normalisation) and oriented so that their normal points away from
    the origin.  Returns float64 vertices and int64 faces.
    """
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    pts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            pts.append((0.0, s1, s2 * phi))
            pts.append((s1, s2 * phi, 0.0))
            pts.append((s2 * phi, 0.0, s1))
    P = np.array(pts, dtype=np.float64)
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    adj = np.abs(d2 - 4.0) < 1e-9
    faces = []
    n = len(P)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    a, b, c = P[i], P[j], P[k]
                    nrm = np.cross(b - a, c - a)
                    if np.dot(nrm, a + b + c) > 0:
                        faces.append((i, j, k))
                    else:
                        faces.append((i, k, j))
    F = np.array(faces, dtype=np.int64)
    assert F.shape == (20, 3)
    V = P / np.linalg.norm(P, axis=1, keepdims=True)
    return V, F


def subdivide(V, F):
    """One 1-to-4 midpoint subdivision with shared (deduplicated) edge midpoints,
    projected back onto the unit sphere.  Orientation is preserved."""
    nv = V.shape[0]
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    key = lo * nv + hi
    uniq, inv = np.unique(key, return_inverse=True)
    ulo = uniq // nv
    uhi = uniq % nv
    mids = 0.5 * (V[ulo] + V[uhi])
    mids /= np.linalg.norm(mids, axis=1, keepdims=True)
    Vn = np.concatenate([V, mids], axis=0)
    nt = F.shape[0]
    m01 = nv + inv[0:nt]
    m12 = nv + inv[nt:2 * nt]
    m20 = nv + inv[2 * nt:3 * nt]
    a, b, c = F[:, 0], F[:, 1], F[:, 2]
    Fn = np.concatenate([
        np.stack([a, m01, m20], 1),
        np.stack([m01, b, m12], 1),
        np.stack([m20, m12, c], 1),
        np.stack([m01, m12, m20], 1),
    ], axis=0)
    return Vn, Fn


def icosphere(level: int):
    """Unit icosphere after ``level`` subdivisions: 20 * 4**level faces (float64)."""
    V, F = icosahedron()
    for _ in range(level):
        V, F = subdivide(V, F)
    return V, F


def _f32(V, F, name, **meta) -> Mesh:
    return Mesh(np.ascontiguousarray(V, dtype=np.float32),
                np.ascontiguousarray(F, dtype=np.int32), name, dict(meta))


def small_cap(level: int = 3, zcut: float = 0.8) -> Mesh:
    """Icosphere of radius 1 with every face whose centroid has z > zcut removed
    (an open cap; the boundary is one loop around the hole)."""
    V, F = icosphere(level)
    V32 = V.astype(np.float32)
    cz = V32[F].astype(np.float64).mean(axis=1)[:, 2]
    F = F[cz <= zcut]
    return _f32(V32, F, f"cap-L{level}", level=level, zcut=zcut)


def displaced_soup(level: int, seed: int, hole_p: float = 0.02,
                   shift=(0.3, 0.0, 0.0), amp: float = 0.05, freq: float = 5.0):
    """Displaced icosphere plus a translated copy, with random faces deleted.

    The unit icosphere vertex v is moved to v * (1 + amp*sin(f x) sin(f y) sin(f z)).
    A second copy is translated by ``shift`` and keeps its own vertex indices, so
    the two shells intersect each other.  Each face is then deleted independently
    with probability ``hole_p`` (first draw of the returned generator), leaving
    holes whose rims form the open boundary.  Returns (mesh, rng) so callers keep
    drawing queries from the same stream.
    """
    V, F = icosphere(level)
    r = 1.0 + amp * np.sin(freq * V[:, 0]) * np.sin(freq * V[:, 1]) * np.sin(freq * V[:, 2])
    V = V * r[:, None]
    V2 = np.concatenate([V, V + np.asarray(shift, dtype=np.float64)[None, :]], axis=0)
    F2 = np.concatenate([F, F + V.shape[0]], axis=0)
    rng = np.random.default_rng(seed)
    keep = rng.random(F2.shape[0]) >= hole_p
    return _f32(V2, F2[keep], f"soup-L{level}", level=level, seed=seed, hole_p=hole_p), rng


# ----------------------------------------------------------------------------
# Queries
# ----------------------------------------------------------------------------

def queries_uniform_bbox(V, n: int, rng, pad: float = 0.1) -> np.ndarray:
    """Uniform points in the vertex bounding box grown by ``pad`` x extent per side."""
    V = np.asarray(V, dtype=np.float64)
    lo, hi = V.min(0), V.max(0)
    ext = hi - lo
    lo = lo - pad * ext
    hi = hi + pad * ext
    return (lo + rng.random((n, 3)) * (hi - lo)).astype(np.float32)


def queries_near_surface(V, F, n: int, rng, sigma: float = 1e-3) -> np.ndarray:
    """Area-weighted uniform surface samples plus isotropic N(0, sigma^2) offsets.

    Draw order: triangle choice, then two uniforms for the barycentric
    coordinates (square-root warp), then the 3 normal offsets per point.
    """
    V = np.asarray(V, dtype=np.float64)
    P = V[F]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    t = np.searchsorted(cdf, rng.random(n), side="right")
    t = np.minimum(t, len(area) - 1)
    r1 = rng.random(n)
    r2 = rng.random(n)
    s = np.sqrt(r1)
    b0 = 1.0 - s
    b1 = s * (1.0 - r2)
    b2 = s * r2
    X = b0[:, None] * P[t, 0] + b1[:, None] * P[t, 1] + b2[:, None] * P[t, 2]
    X += rng.normal(0.0, sigma, size=(n, 3))
    return X.astype(np.float32)


def grid_queries(V, res: int, pad: float = 0.1) -> np.ndarray:
    """Cell centres of a res^3 grid over the padded bounding box (x fastest)."""
    V = np.asarray(V, dtype=np.float64)
    lo, hi = V.min(0), V.max(0)
    ext = hi - lo
    lo = lo - pad * ext
    hi = hi + pad * ext
    c = [(lo[d] + (np.arange(res) + 0.5) * (hi[d] - lo[d]) / res) for d in range(3)]
    z, y, x = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float32)


# ----------------------------------------------------------------------------
# Precision / robustness workload (integer geometry)
# ----------------------------------------------------------------------------

_CUBE_FACES = {
    # axis, side -> quad corners (as offsets from the voxel's min corner), CCW seen
    # from outside of the voxel along the face's outward normal.
    (0, 0): [(0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)],
    (0, 1): [(1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)],
    (1, 0): [(0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)],
    (1, 1): [(0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)],
    (2, 0): [(0, 0, 0), (0, 1, 0), (1, 1, 0), (1, 0, 0)],
    (2, 1): [(0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)],
}


def _check_cube_faces():
    for (axis, side), quad in _CUBE_FACES.items():
        q = np.array(quad, dtype=np.float64)
        nrm = np.cross(q[1] - q[0], q[2] - q[0])
        out = np.zeros(3)
        out[axis] = 1.0 if side else -1.0
        assert np.dot(nrm, out) > 0, (axis, side)


def staircase_sphere(radius: float = 40.0) -> Mesh:
    """Closed voxel staircase: the boundary faces of all unit voxels whose centre
    lies strictly inside the sphere of ``radius`` (integer grid, welded by
    coordinate, outward orientation, each quad split along its 0-2 diagonal)."""
    _check_cube_faces()
    R = int(math.ceil(radius)) + 1
    ax = np.arange(-R, R)
    I, J, K = np.meshgrid(ax, ax, ax, indexing="ij")
    c2 = (I + 0.5) ** 2 + (J + 0.5) ** 2 + (K + 0.5) ** 2
    inside = c2 < radius * radius
    quads = []
    for (axis, side), quad in _CUBE_FACES.items():
        step = np.zeros(3, dtype=int)
        step[axis] = 1 if side else -1
        nb = np.roll(inside, shift=-step[axis], axis=axis)
        mask = inside & ~nb
        idx = np.argwhere(mask)
        base = ax[idx]
        corners = np.stack([base + np.array(off) for off in quad], axis=1)  # [m,4,3]
        quads.append(corners)
    Q = np.concatenate(quads, axis=0)
    pts = Q.reshape(-1, 3)
    uniq, inv = np.unique(pts, axis=0, return_inverse=True)
    inv = inv.reshape(-1, 4)
    F = np.concatenate([inv[:, [0, 1, 2]], inv[:, [0, 2, 3]]], axis=0)
    return _f32(uniq, F, f"staircase-r{radius:g}", radius=radius, quads=int(Q.shape[0]))


def height_field_patch(rng, n: int = 200, z0: int = 45, dz: int = 3, x0: int = -100) -> Mesh:
    """Open n x n height field at integer (x, y) in [x0, x0+n-1]^2 with integer
    heights z0 + U{-dz..dz}; cells split along the (i,j)-(i+1,j+1) diagonal, normals up."""
    h = z0 + rng.integers(-dz, dz + 1, size=(n, n))
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")  # ii ~ x, jj ~ y
    V = np.stack([x0 + ii, x0 + jj, h], -1).reshape(-1, 3).astype(np.float64)
    vid = lambda i, j: i * n + j
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    i = i.ravel(); j = j.ravel()
    a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    return _f32(V, F, f"heightfield-{n}", n=n)


def _merge(meshes, name):
    Vs, Fs, off = [], [], 0
    for m in meshes:
        Vs.append(m.V.astype(np.float64))
        Fs.append(m.F.astype(np.int64) + off)
        off += m.nv
    return _f32(np.concatenate(Vs), np.concatenate(Fs), name)


def precision_workload(n_query: int = 500_000, seed: int = 2, radius: float = 40.0):
    """Voxel staircase of a sphere plus an open integer height field above it.

    Queries, n_query/4 of each kind, all exactly representable in FP32:
    random mesh vertices; midpoints of random mesh edges; points on random
    axis-aligned staircase faces (the face's coordinate is an integer, the two
    in-face coordinates are multiples of 1/8 inside the unit square); integer
    grid points in the bounding box.  Draw order: patch heights, then the four
    kinds in that order.
    """
    rng = np.random.default_rng(seed)
    st = staircase_sphere(radius)
    patch = height_field_patch(rng)
    mesh = _merge([st, patch], "precision")
    mesh.meta.update(staircase_tris=st.nt, patch_tris=patch.nt)
    k = n_query // 4
    V = mesh.V.astype(np.float64)
    q1 = V[rng.integers(0, mesh.nv, size=k)]
    tri = rng.integers(0, mesh.nt, size=k)
    e = rng.integers(0, 3, size=k)
    va = mesh.F[tri, e]
    vb = mesh.F[tri, (e + 1) % 3]
    q2 = 0.5 * (V[va] + V[vb])
    stF = st.F
    ft = rng.integers(0, st.nt, size=k)
    P = st.V.astype(np.float64)[stF[ft]]          # [k,3,3]
    lo = P.min(1)
    hi = P.max(1)
    flat = np.argmin(hi - lo, axis=1)            # the axis of the face plane
    u = rng.integers(0, 9, size=(k, 3)) / 8.0
    q3 = lo + u * (hi - lo)
    q3[np.arange(k), flat] = lo[np.arange(k), flat]
    bl = np.floor(V.min(0)) - 1
    bh = np.ceil(V.max(0)) + 1
    q4 = rng.integers(bl.astype(np.int64), bh.astype(np.int64) + 1, size=(k, 3)).astype(np.float64)
    Q = np.concatenate([q1, q2, q3, q4]).astype(np.float32)
    kinds = np.repeat(np.arange(4, dtype=np.int8), k)
    return mesh, Q, kinds


# ----------------------------------------------------------------------------
# Batched workload: superquadrics, height fields and soups
# ----------------------------------------------------------------------------

def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def superquadric(n_tri_target: int, e1: float, e2: float, rng) -> Mesh:
    """Closed superquadric (exponents e1, e2) on a latitude/longitude grid, welded
    at the seam and the poles, outward orientation, random scale/rotation/offset."""
    nu = max(3, int(round(math.sqrt(n_tri_target / 2.0))))
    nvv = max(2, int(round(n_tri_target / (2.0 * nu))))
    def spow(c, e):
        return np.sign(c) * np.abs(c) ** e
    eta = -math.pi / 2 + math.pi * np.arange(1, nvv) / nvv     # interior rings
    om = 2 * math.pi * np.arange(nu) / nu
    E, O = np.meshgrid(eta, om, indexing="ij")
    X = spow(np.cos(E), e1) * spow(np.cos(O), e2)
    Y = spow(np.cos(E), e1) * spow(np.sin(O), e2)
    Z = spow(np.sin(E), e1)
    ring = np.stack([X, Y, Z], -1).reshape(-1, 3)
    south = np.array([[0.0, 0.0, -1.0]])
    north = np.array([[0.0, 0.0, 1.0]])
    V = np.concatenate([ring, south, north])
    nr = nvv - 1
    s_id = nr * nu
    n_id = s_id + 1
    vid = lambda r, c: r * nu + (c % nu)
    F = []
    c = np.arange(nu)
    F.append(np.stack([np.full(nu, s_id), vid(0, c + 1), vid(0, c)], 1))
    for r in range(nr - 1):
        a, b, cc, d = vid(r, c), vid(r, c + 1), vid(r + 1, c + 1), vid(r + 1, c)
        F.append(np.stack([a, b, cc], 1))
        F.append(np.stack([a, cc, d], 1))
    F.append(np.stack([vid(nr - 1, c), vid(nr - 1, c + 1), np.full(nu, n_id)], 1))
    F = np.concatenate(F)
    # orient outward (check one face well away from the poles)
    P = V[F]
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    if np.sum(np.einsum("ij,ij->i", nrm, P.mean(1))) < 0:
        F = F[:, [0, 2, 1]]
    scale = rng.uniform(0.5, 2.0, size=3)
    V = (V * scale) @ _rotation(rng).T + rng.uniform(-1, 1, size=3)
    return _f32(V, F, "superquadric", e1=e1, e2=e2)


def queries_near_triangle_edges(V, F, n: int, rng, lo: float = -6.0, hi: float = -4.5) -> np.ndarray:
    """Points just off the interior of triangle edges.

    Draw order: n distinct triangles, the edge of each (0-1, 1-2, 2-0), the
    parameter along it (U[0.2, 0.8]), a normal direction made perpendicular
    to the edge, and the distance as 10^U[lo, hi] edge lengths.  In an
    unwelded soup every such edge is a boundary edge.
    """
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F)
    tri = rng.choice(len(F), n, replace=False)
    k = rng.integers(0, 3, n)
    a = V[F[tri, k]]
    b = V[F[tri, (k + 1) % 3]]
    t = rng.uniform(0.2, 0.8, n)[:, None]
    off = rng.normal(size=(n, 3))
    e = b - a
    off -= (np.sum(off * e, 1) / np.sum(e * e, 1))[:, None] * e
    off /= np.linalg.norm(off, axis=1)[:, None]
    dist = 10.0 ** rng.uniform(lo, hi, n) * np.linalg.norm(e, axis=1)
    return (a + t * e + dist[:, None] * off).astype(np.float32)


def random_soup(n_tri: int, rng) -> Mesh:
    """Unwelded random triangles in the unit cube, edge length ~ U[0.01, 0.2]."""
    c = rng.random((n_tri, 3))
    L = rng.uniform(0.01, 0.2, size=n_tri)
    d1 = rng.normal(size=(n_tri, 3)); d1 /= np.linalg.norm(d1, axis=1, keepdims=True)
    d2 = rng.normal(size=(n_tri, 3)); d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
    p0 = c
    p1 = c + L[:, None] * d1
    p2 = c + L[:, None] * d2
    V = np.stack([p0, p1, p2], 1).reshape(-1, 3)
    F = np.arange(3 * n_tri).reshape(-1, 3)
    return _f32(V, F, "soup")


def random_height_field(n_tri_target: int, rng) -> Mesh:
    n = max(2, int(round(math.sqrt(n_tri_target / 2.0))) + 1)
    h = 0.1 * rng.normal(size=(n, n))
    xs = np.linspace(0, 1, n)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    V = np.stack([xs[ii], xs[jj], h], -1).reshape(-1, 3)
    vid = lambda i, j: i * n + j
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    i = i.ravel(); j = j.ravel()
    a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0)
    V = V @ _rotation(rng).T
    return _f32(V, F, "heightfield")


def batched_workload(n_mesh: int = 256, seed: int = 3, tri_range=(100, 500_000),
                     q_range=(1_000, 1_000_000), scale: float = 1.0):
    """Many meshes of uneven sizes with uneven query sets.

    Kinds cycle superquadric / height field / soup.  Triangle and query counts are
    log-uniform in the given ranges (multiplied by ``scale`` for reduced test
    sizes); half the queries of each mesh are uniform in its padded bbox and half
    near its surface.  Returns a list of (mesh, queries).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_mesh):
        kind = i % 3
        nt = int(round(math.exp(rng.uniform(math.log(tri_range[0]), math.log(tri_range[1]))) * scale))
        nq = int(round(math.exp(rng.uniform(math.log(q_range[0]), math.log(q_range[1]))) * scale))
        nt = max(nt, 4)
        nq = max(nq, 2)
        if kind == 0:
            m = superquadric(nt, rng.uniform(0.3, 3.0), rng.uniform(0.3, 3.0), rng)
        elif kind == 1:
            m = random_height_field(nt, rng)
        else:
            m = random_soup(nt, rng)
        q = np.concatenate([queries_uniform_bbox(m.V, nq // 2, rng),
                            queries_near_surface(m.V, m.F, nq - nq // 2, rng)])
        out.append((m, q))
    return out


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def workload(name: str, n_query: int | None = None):
    """Named workloads used by the tests and the benchmark.

    ``small``: icosphere level 3 with the z>0.8 cap removed; 10,000 uniform
    queries in [-1.5, 1.5]^3 (seed 0).
    ``soup7``: displaced level-7 icosphere + translated copy, 2% holes; 1M
    uniform-in-padded-bbox + 1M near-surface queries (seed 1).
    ``soup8``: the same at level 8 (the ~1M-triangle-per-shell mesh, 2.57M
    triangles in total); 1M + 1M queries (seed 4).
    ``precision``: voxel-staircase sphere (radius 40) + integer height field;
    500k queries on vertices, edge midpoints, faces and grid points (seed 2).
    ``n_query`` overrides the total query count (split evenly).
    Returns (mesh, Q).
    """
    if name == "small":
        m = small_cap(3, 0.8)
        rng = np.random.default_rng(0)
        n = 10_000 if n_query is None else n_query
        Q = (-1.5 + 3.0 * rng.random((n, 3))).astype(np.float32)
        return m, Q
    if name in ("soup7", "soup8"):
        level, seed = (7, 1) if name == "soup7" else (8, 4)
        m, rng = displaced_soup(level, seed)
        n = 2_000_000 if n_query is None else n_query
        Q = np.concatenate([queries_uniform_bbox(m.V, n // 2, rng),
                            queries_near_surface(m.V, m.F, n - n // 2, rng)])
        return m, Q
    if name == "precision":
        m, Q, _ = precision_workload(500_000 if n_query is None else n_query)
        return m, Q
    raise KeyError(name)


# ----------------------------------------------------------------------------
# Parametric surfaces (Sec. 4.4): bicubic Bezier patches
# ----------------------------------------------------------------------------

def bezier_patches(n_patch: int = 100, seed: int = 7) -> np.ndarray:
    """``n_patch`` bicubic Bezier patches whose 16 control points are each uniform
    in the unit cube (the paper's random-patch benchmark, Sec. 5): float32
    ``[n_patch, 4, 4, 3]``, C[p][i][j] with i along u and j along v.  Draws
    ``n_patch * 48`` uniforms from one PCG64 stream."""
    rng = np.random.default_rng(seed)
    return rng.random((n_patch, 4, 4, 3)).astype(np.float32)


def param_workload(res: int = 32, n_patch: int = 100, seed: int = 7):
    """(patches, Q): :func:`bezier_patches` and the cell centres of a res^3 grid
    over the control points' bounding box padded by 10% per side (x fastest),
    the voxelization scenario of the parametric benchmark."""
    P = bezier_patches(n_patch, seed)
    return P, grid_queries(P.reshape(-1, 3), res)


def surrogate_workload(level: int = 8, n_train: int = 2_000_000, res: int = 256, seed: int = 4):
    """The learned-surrogate workload: the displaced, self-intersecting, holed
    soup at ``level`` (seed ``seed``), ``n_train`` training samples (half
    uniform in the bbox padded by 10%, half near-surface) and the ``res``^3
    grid of cell centres over the padded bbox.  Returns (mesh, samples, grid)."""
    m, rng = displaced_soup(level, seed)
    S = np.concatenate([queries_uniform_bbox(m.V, n_train // 2, rng),
                        queries_near_surface(m.V, m.F, n_train - n_train // 2, rng)])
    return m, S, grid_queries(m.V, res)
