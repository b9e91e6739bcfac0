"""Pins of the oracle's boundary extraction and antipodal evaluation (no GPU).

* ``oracle.boundary`` against a Counter-based net multiplicity on random meshes,
  closed meshes (empty boundary), soups (B = 3F) and the boundary being a 1-cycle
  (in-degree = out-degree at every vertex), Sec. 4.1.
* ``oracle.antipodal`` (Eq. 9 with x1 = -z) against the direct sum (Eq. 2):
  equal to 1e-10 off the surface (Sec. 4.1), including queries whose vertical ray
  passes exactly through a boundary vertex (the perturbation limit) and the
  grazing-ray neighbourhood of the paper's robustness figure (Supp. S2), where no
  integer jump may appear; and 1e-6 to 3e-5 edge lengths from boundary edges of
  a soup, the ill-conditioned regime the GPU's FP64 re-evaluation of cancelling
  terms is judged in (the two formulas round differently there, so agreement to
  1e-9 bounds the oracle's own error).
* Independence of the ray direction (Algorithm 1 picks x0 arbitrarily): a numpy
  re-implementation of Algorithm 1 with random directions x0, its crossing number
  found by generic ray casting, gives the same w.
* Queries on the surface but off the boundary: w(q_eps) is the limit from the
  side the perturbation picks.
"""
from collections import Counter

import numpy as np
import pytest

import gen
import oracle


def _boundary_counter(F):
    c = Counter()
    for t in F:
        for e in range(3):
            u, v = int(t[e]), int(t[(e + 1) % 3])
            if u == v:
                continue
            if u < v:
                c[(u, v)] += 1
            else:
                c[(v, u)] -= 1
    out = []
    for (u, v), m in c.items():
        out += [(u, v)] * m if m > 0 else [(v, u)] * (-m)
    return sorted(out)


def test_boundary_against_counter():
    rng = np.random.default_rng(0)
    for trial in range(30):
        nv = int(rng.integers(3, 12))
        nt = int(rng.integers(1, 40))
        F = np.stack([rng.choice(nv, 3, replace=False) for _ in range(nt)]).astype(np.int32)
        if trial % 3 == 0:   # degenerate faces with a repeated index
            F[: nt // 2, 1] = F[: nt // 2, 0]
        E = oracle.boundary(F, nv)
        assert sorted(map(tuple, E.tolist())) == _boundary_counter(F)


def test_boundary_special_cases():
    V, F = gen.icosphere(2)
    assert len(oracle.boundary(F.astype(np.int32), len(V))) == 0
    soup = gen.random_soup(50, np.random.default_rng(1))
    assert len(oracle.boundary(soup.F, soup.nv)) == 150
    # one triangle
    assert sorted(map(tuple, oracle.boundary(np.array([[0, 1, 2]], np.int32), 3).tolist())) == [(0, 1), (1, 2), (2, 0)]
    # two triangles glued with inconsistent orientation: the shared edge counts twice
    E = oracle.boundary(np.array([[0, 1, 2], [0, 1, 3]], np.int32), 4)
    assert len(E) == 6 and sum(1 for e in E.tolist() if tuple(e) == (0, 1)) == 2
    m = gen.displaced_soup(3, seed=5)[0]
    E = oracle.boundary(m.F, m.nv)
    deg_out = np.bincount(E[:, 0], minlength=m.nv)
    deg_in = np.bincount(E[:, 1], minlength=m.nv)
    assert np.array_equal(deg_in, deg_out)


@pytest.mark.parametrize("name", ["small", "soup3"])
def test_antipodal_equals_direct_off_surface(name):
    if name == "small":
        m, Q = gen.workload("small", n_query=3000)
    else:
        m, rng = gen.displaced_soup(3, seed=9)
        Q = np.concatenate([gen.queries_uniform_bbox(m.V, 1500, rng),
                            gen.queries_near_surface(m.V, m.F, 1500, rng)])
    r = oracle.reference(m.V, m.F, Q, with_direct=True)
    assert np.all(r["flags"] == 0)
    assert np.max(np.abs(r["w_antipodal"] - r["w_direct"])) < 1e-10


@pytest.mark.parametrize("seed", [11, 12])
def test_antipodal_equals_direct_near_boundary_edges(seed):
    rng = np.random.default_rng(seed)
    m = gen.random_soup(400, rng)
    Q = gen.queries_near_triangle_edges(m.V, m.F, 64, rng)
    r = oracle.reference(m.V, m.F, Q, with_direct=True)
    ok = r["flags"] == 0
    assert ok.sum() >= 48
    # FP64 rounding amplified by at most ~1e6 (edge length over distance) per term
    assert np.max(np.abs(r["w_antipodal"] - r["w_direct"])[ok]) < 1e-9


def test_ray_through_boundary_vertex():
    """Queries straight below (and above) every boundary vertex of the open cap:
    the crossing test and the boundary term both take the perturbation limit."""
    m = gen.small_cap(3, 0.8)
    E = oracle.boundary(m.F, m.nv)
    bv = np.unique(E.ravel())
    P = m.V[bv]
    Q = []
    for z in (-1.3, -0.5, 0.0, 0.5, 0.7, 1.4):
        Qk = P.copy()
        Qk[:, 2] = z
        Q.append(Qk)
    Q = np.concatenate(Q).astype(np.float32)
    r = oracle.reference(m.V, m.F, Q, with_direct=True)
    assert np.all(r["flags"] == 0)
    assert np.max(np.abs(r["w_antipodal"] - r["w_direct"])) < 1e-10


def test_grazing_square_has_no_integer_jumps():
    """The robustness figure of Supp. S2: queries on a grid inside a 1e-6 square
    around a point whose vertical ray grazes a boundary edge and a boundary vertex
    of an open mesh; w must be continuous (equal to the direct sum)."""
    m = gen.small_cap(3, 0.8)
    E = oracle.boundary(m.F, m.nv)
    a, b = m.V[E[0, 0]].astype(np.float64), m.V[E[0, 1]].astype(np.float64)
    Q = []
    for centre in (a, 0.5 * (a + b)):
        xs = centre[0] + np.linspace(-5e-7, 5e-7, 21)
        ys = centre[1] + np.linspace(-5e-7, 5e-7, 21)
        X, Y = np.meshgrid(xs, ys)
        Q.append(np.stack([X.ravel(), Y.ravel(), np.full(X.size, -0.2)], 1))
    Q = np.concatenate(Q).astype(np.float32)
    r = oracle.reference(m.V, m.F, Q, with_direct=True)
    d = np.abs(r["w_antipodal"] - r["w_direct"])
    # no integer (or any large) jump; the residue is FP64 rounding of the unit
    # vectors, amplified near the pole by 1/(angle to the vertex) ~ 1e7
    assert np.max(d) < 1e-7
    # the region really straddles the jump of chi
    assert len(np.unique(r["chi"])) >= 2


def _alg1_random_direction(V, F, E, Q, x0):
    """Algorithm 1 with an arbitrary direction x0 in plain numpy: chi by
    Moller-Trumbore ray casting along x0, area term with the pole x1 = -x0."""
    V = V.astype(np.float64)
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1, e2 = B - A, C - A
    nrm = np.cross(e1, e2)
    out = []
    x1 = -x0
    for q in Q.astype(np.float64):
        p = np.cross(x0, e2)
        det = np.einsum("ij,ij->i", e1, p)
        inv = 1.0 / det
        s = q - A
        u = np.einsum("ij,ij->i", s, p) * inv
        qq = np.cross(s, e1)
        v = (qq @ x0) * inv
        t = np.einsum("ij,ij->i", e2, qq) * inv
        hit = (u > 0) & (v > 0) & (u + v < 1) & (t > 0)
        chi = int(np.sum(np.sign(nrm[hit] @ x0)))
        a = V[E[:, 0]] - q
        b = V[E[:, 1]] - q
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        b /= np.linalg.norm(b, axis=1, keepdims=True)
        num = np.einsum("ij,ij->i", a, np.cross(b, x1[None, :]))
        den = 1 + np.einsum("ij,ij->i", a, b) + a @ x1 + b @ x1
        out.append(chi + np.sum(2 * np.arctan2(num, den)) / (4 * np.pi))
    return np.array(out)


def test_direction_independence():
    m, Q = gen.workload("small", n_query=300)
    E = oracle.boundary(m.F, m.nv)
    w_ref = oracle.direct(m.V, m.F, Q)
    rng = np.random.default_rng(12)
    for _ in range(3):
        x0 = rng.normal(size=3)
        x0 /= np.linalg.norm(x0)
        w = _alg1_random_direction(m.V, m.F, E, Q, x0)
        assert np.max(np.abs(w - w_ref)) < 1e-9


def test_on_surface_queries_take_the_perturbed_side():
    """For queries exactly on faces of the open integer height field (not on its
    boundary), w(q_eps) equals the direct sum just above or below the face, on
    the side the perturbation (+e1, +e2, +e3) selects."""
    rng = np.random.default_rng(21)
    m = gen.height_field_patch(rng, n=12, z0=0, dz=2, x0=0)
    E = oracle.boundary(m.F, m.nv)
    V = m.V.astype(np.float64)
    t = rng.integers(0, m.nt, 400)
    bary = rng.integers(1, 7, (400, 3)).astype(np.float64)
    bary /= bary.sum(1, keepdims=True)
    Q = np.einsum("ij,ijk->ik", bary, V[m.F[t]])
    # keep only exactly representable points
    Q32 = Q.astype(np.float32)
    ok = np.all(Q32.astype(np.float64) == Q, axis=1)
    Q32 = Q32[ok]
    chi = oracle.chi(m.V, m.F, Q32)
    w, fl = oracle.antipodal(m.V, E, Q32, chi)
    assert np.all(fl == 0)
    off = np.array([1e-3, 1e-5, 1e-7])
    wp = oracle.direct(m.V, m.F, (Q32.astype(np.float64) + off).astype(np.float32))
    assert np.max(np.abs(w - wp)) < 2e-2
    assert len(Q32) > 50
