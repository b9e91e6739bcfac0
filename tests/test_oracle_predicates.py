"""Pins of the oracle's exact, symbolically perturbed crossing predicates (no GPU).

The oracle evaluates the 2-D edge classification, the supporting-plane side and
the ray-triangle crossing of Supp. S2.1 on big integers with the lexicographic
(real, e1, e2, e3) rule.  These tests check it against a different formulation
evaluated in exact rational arithmetic at an actual perturbed point
q + (2^-40, 2^-80, 2^-120) on small integer inputs (where that point is
infinitesimally close in the sense of the perturbation order): the ray's
intersection parameter t and the barycentric coordinates of the hit point.
They also pin the crossing count on a closed mesh against the integer winding
number at a perturbed, off-surface point, including queries placed exactly on
vertices, edges and faces.
"""
import itertools
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import gen
import oracle

EPS = (Fr(1, 2 ** 40), Fr(1, 2 ** 80), Fr(1, 2 ** 120))
EPS_SMALLER = (Fr(1, 2 ** 60), Fr(1, 2 ** 120), Fr(1, 2 ** 180))


def _sign(x):
    return (x > 0) - (x < 0)


def _perturbed(q, eps):
    return [Fr(float(q[0])) + eps[0], Fr(float(q[1])) + eps[1], Fr(float(q[2])) + eps[2]]


def _edge_brute(q, pi, pj, eps):
    x, y, _ = _perturbed(q, eps)
    xi, yi, xj, yj = (Fr(float(v)) for v in (pi[0], pi[1], pj[0], pj[1]))
    return _sign((x - xi) * (yi - yj) + (y - yi) * (xj - xi))


def _crossing_brute(q, a, b, c, eps):
    """Ray p + t(0,0,1), p the perturbed query: +-1 when it hits the triangle at
    t > 0 with all barycentric coordinates of the hit point positive."""
    p = _perturbed(q, eps)
    A, B, C = ([Fr(float(v)) for v in P] for P in (a, b, c))
    u = [B[k] - A[k] for k in range(3)]
    v = [C[k] - A[k] for k in range(3)]
    n = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]
    if n[2] == 0:
        return 0
    t = sum(n[k] * (A[k] - p[k]) for k in range(3)) / n[2]
    if t <= 0:
        return 0
    hx, hy = p[0], p[1]
    # barycentric coordinates of (hx, hy) in the projected triangle
    det = (B[0] - A[0]) * (C[1] - A[1]) - (C[0] - A[0]) * (B[1] - A[1])
    l1 = ((hx - A[0]) * (C[1] - A[1]) - (C[0] - A[0]) * (hy - A[1])) / det
    l2 = ((B[0] - A[0]) * (hy - A[1]) - (hx - A[0]) * (B[1] - A[1])) / det
    l0 = 1 - l1 - l2
    if l0 > 0 and l1 > 0 and l2 > 0:
        return _sign(n[2])
    return 0


def _small_int_cases(seed, n, lo=-2, hi=2):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield rng.integers(lo, hi + 1, size=(4, 3)).astype(np.float32)


def test_edge_sign_matches_rational_brute_force():
    for P in _small_int_cases(1, 3000):
        q, a, b = P[0], P[1], P[2]
        got = oracle.edge_sos(q, a, b)
        if a[0] == b[0] and a[1] == b[1]:
            assert got == 0
            continue
        assert got == _edge_brute(q, a, b, EPS) == _edge_brute(q, a, b, EPS_SMALLER)
        # antisymmetry under edge reversal, which makes shared edges watertight
        assert oracle.edge_sos(q, b, a) == -got


def test_crossing_matches_rational_brute_force():
    hits = 0
    for P in _small_int_cases(2, 6000):
        q, a, b, c = P
        got = oracle.tri_crossing(q, a, b, c)
        ref = _crossing_brute(q, a, b, c, EPS)
        assert got == ref == _crossing_brute(q, a, b, c, EPS_SMALLER), (P, got, ref)
        hits += got != 0
    assert hits > 200


def test_crossing_with_fractional_coordinates():
    # half-integer and quarter coordinates, still exact in FP32
    rng = np.random.default_rng(3)
    for _ in range(3000):
        P = (rng.integers(-8, 9, size=(4, 3)) / 4.0).astype(np.float32)
        q, a, b, c = P
        assert oracle.tri_crossing(q, a, b, c) == _crossing_brute(q, a, b, c, EPS)


def test_plane_side_matches_rational_brute_force():
    for P in _small_int_cases(4, 3000):
        q, a, b, c = P
        p = _perturbed(q, EPS)
        A, B, C = ([Fr(float(v)) for v in X] for X in (a, b, c))
        u = [B[k] - A[k] for k in range(3)]
        v = [C[k] - A[k] for k in range(3)]
        n = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]
        ref = _sign(sum(n[k] * (A[k] - p[k]) for k in range(3)))
        assert oracle.plane_sos(q, a, b, c) == ref


def test_shared_edge_counted_once():
    # a ray through the common edge of two coplanar triangles of the square
    # [0,2]^2 crosses exactly once; on the square's own rim the perturbation
    # (+e1, +e2) decides: the left and bottom sides are in, right and top out
    V = np.array([[0, 0, 1], [2, 0, 1], [2, 2, 1], [0, 2, 1]], dtype=np.float32)
    tris = [(0, 1, 2), (0, 2, 3)]
    cases = {(1, 1, 0): 1, (0.5, 0.5, 0): 1, (1.5, 1.5, -7): 1, (0, 0, 0): 1,
             (0, 1, 0): 1, (1, 0, 0): 1, (2, 2, -3): 0, (2, 1, 0): 0, (1, 2, 0): 0,
             (0, 2, 0): 0, (2, 0, 0): 0, (1, 1, 1): 0, (1, 1, 2): 0}
    for q, want in cases.items():
        q = np.array(q, dtype=np.float32)
        total = sum(oracle.tri_crossing(q, V[i], V[j], V[k]) for i, j, k in tris)
        assert total == want, q


def test_closed_staircase_chi_equals_winding_at_perturbed_point():
    """On the closed voxel staircase every query kind (vertices, edge midpoints,
    face points, grid points) gets chi equal to the integer winding number at
    q + (1/128, 1/1024, 1/8192).  Coordinates are multiples of 1/8 and the mesh is
    unit-grid axis-aligned, so that offset lies on the same side of every
    predicate as the infinitesimal perturbation (the real part is a nonzero
    multiple of 1/8 or zero, and each perturbation coefficient is 0 or +-1)."""
    st = gen.staircase_sphere(6.0)
    rng = np.random.default_rng(7)
    V = st.V.astype(np.float64)
    k = 150
    q1 = V[rng.integers(0, st.nv, k)]
    t = rng.integers(0, st.nt, k)
    e = rng.integers(0, 3, k)
    q2 = 0.5 * (V[st.F[t, e]] + V[st.F[t, (e + 1) % 3]])
    t = rng.integers(0, st.nt, k)
    P = V[st.F[t]]
    lo, hi = P.min(1), P.max(1)
    flat = np.argmin(hi - lo, 1)
    q3 = lo + rng.integers(0, 9, (k, 3)) / 8.0 * (hi - lo)
    q3[np.arange(k), flat] = lo[np.arange(k), flat]
    q4 = rng.integers(-8, 9, (k, 3)).astype(np.float64)
    Q = np.concatenate([q1, q2, q3, q4]).astype(np.float32)
    off = np.array([1 / 128, 1 / 1024, 1 / 8192])
    Qp = (Q.astype(np.float64) + off).astype(np.float32)
    assert np.all(Qp.astype(np.float64) == Q.astype(np.float64) + off)
    chi = oracle.chi(st.V, st.F, Q)
    w = oracle.direct(st.V, st.F, Qp)
    assert np.max(np.abs(w - np.round(w))) < 1e-9
    assert np.array_equal(chi, np.round(w).astype(np.int32))
    assert set(np.unique(chi)) <= {0, 1}
    assert 0 < chi.sum() < len(chi)
