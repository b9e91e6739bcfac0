"""Pins of ``oracle.gradient`` (Supp. S4, Algorithm 3) to facts other than itself.

* Finite differences of the oracle's antipodal w (Eq. 9, pinned by its own
  closed-form tests): Richardson-extrapolated central differences at queries
  whose six stencil points share the crossing count (w is smooth there).
* The disk on its axis: w = -(1/4pi) 2pi (1 - |h| / sqrt(h^2 + R^2)) sgn(h) for a
  fan-triangulated N-gon (normal +z) seen from height h, so
  dw/dh = +(1/2) R^2 / (h^2 + R^2)^(3/2) on both sides, and the x, y
  components vanish by symmetry.
* Direction independence: the crossing count is piecewise constant for every
  ray direction, so the gradient of the boundary terms cannot depend on the
  antipode x1 (Supp. S4); random x1 must give the -z result.
* A closed mesh has no boundary and a zero gradient.
"""
import math

import numpy as np
import pytest

import gen
import oracle


def _fd_gradient(V, E, F, q, h):
    """Central differences of the antipodal w (its chi from the same stencil point)."""
    g = np.zeros(3)
    chis = []
    for k in range(3):
        vals = []
        for s in (+1, -1):
            p = q.astype(np.float64).copy()
            p[k] += s * h
            P = p.astype(np.float32)[None, :]
            assert P[0, k] == p[k]          # the step is exact in FP32
            c = oracle.chi(V, F, P)
            chis.append(int(c[0]))
            w, fl = oracle.antipodal(V, E, P, c)
            assert fl[0] == 0
            vals.append(w[0])
        g[k] = (vals[0] - vals[1]) / (2 * h)
    return g, len(set(chis)) == 1


def _richardson(V, E, F, q, h):
    g1, ok1 = _fd_gradient(V, E, F, q, h)
    g2, ok2 = _fd_gradient(V, E, F, q, h / 2)
    return (4 * g2 - g1) / 3, ok1 and ok2


@pytest.mark.parametrize("name", ["cap", "soup"])
def test_gradient_matches_finite_differences(name):
    if name == "cap":
        m = gen.small_cap(3, 0.8)
    else:
        m, _ = gen.displaced_soup(2, seed=5, hole_p=0.1)
    E = oracle.boundary(m.F, m.nv)
    assert len(E) > 0
    rng = np.random.default_rng(7)
    # queries on a grid of multiples of 2^-6 so that q +- h stays exact in FP32
    Q = (np.round(rng.uniform(-1.4, 1.4, size=(60, 3)) * 64) / 64).astype(np.float32)
    g, a, c, fl = oracle.gradient(m.V, E, Q)
    checked = 0
    for i in range(len(Q)):
        if fl[i]:
            continue
        fd, smooth = _richardson(m.V, E, m.F, Q[i], 2.0 ** -10)
        if not smooth:
            continue     # the stencil crosses the surface: w jumps there
        tol = 1e-6 * (1.0 + c[i])
        assert np.all(np.abs(fd - g[i]) <= tol), (i, Q[i], fd, g[i], c[i])
        checked += 1
    assert checked >= 40


@pytest.mark.parametrize("h", [0.25, 1.0, 3.0, -0.5, -2.0])
def test_disk_on_axis(h):
    N, R = 2048, 1.0
    t = 2 * np.pi * np.arange(N) / N
    V = np.concatenate([[[0.0, 0.0, 0.0]], np.stack([R * np.cos(t), R * np.sin(t), np.zeros(N)], 1)])
    F = np.array([[0, 1 + i, 1 + (i + 1) % N] for i in range(N)], np.int32)   # normal +z
    V = V.astype(np.float32)
    E = oracle.boundary(F, len(V))
    assert len(E) == N
    g, a, c, fl = oracle.gradient(V, E, np.array([[0.0, 0.0, h]], np.float32))
    # the inscribed N-gon has area (N/2) sin(2 pi / N) R^2 instead of pi R^2: relative
    # change of order (2 pi / N)^2 / 6 in every moment of the rim
    want = 0.5 * R * R / (h * h + R * R) ** 1.5
    assert abs(g[0, 2] - want) <= 1e-5 * abs(want), (g[0], want)
    assert abs(g[0, 0]) < 1e-12 and abs(g[0, 1]) < 1e-12
    # the same sign convention as w itself: w(h) = -(1/2)(1 - |h| / sqrt(h^2 + R^2)) sgn(h)
    c0 = oracle.chi(V, F, np.array([[0.0, 0.0, h]], np.float32))
    w, _ = oracle.antipodal(V, E, np.array([[0.0, 0.0, h]], np.float32), c0)
    w_disk = -0.5 * (1.0 - abs(h) / math.sqrt(h * h + R * R)) * math.copysign(1.0, h)
    assert abs(w[0] - w_disk) < 1e-5


def test_direction_independence():
    m, _ = gen.displaced_soup(2, seed=8, hole_p=0.1)
    E = oracle.boundary(m.F, m.nv)
    rng = np.random.default_rng(9)
    Q = rng.uniform(-1.3, 1.3, size=(50, 3)).astype(np.float32)
    g0, a0, c0, f0 = oracle.gradient(m.V, E, Q)
    for _ in range(4):
        x1 = rng.normal(size=3)
        x1 /= np.linalg.norm(x1)
        g1, a1, c1, f1 = oracle.gradient(m.V, E, Q, x1=x1)
        ok = (f0 == 0) & (f1 == 0)
        tol = 1e-9 * (1.0 + np.maximum(c0, c1))
        assert np.all(np.abs(g1 - g0)[ok] <= tol[ok, None])


def test_closed_mesh_has_zero_gradient():
    V, F = gen.icosphere(2)
    E = oracle.boundary(F.astype(np.int32), len(V))
    assert len(E) == 0
    g, a, c, fl = oracle.gradient(V.astype(np.float32), E, np.zeros((3, 3), np.float32))
    assert np.all(g == 0)
