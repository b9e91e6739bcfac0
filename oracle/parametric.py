"""Float64 reference for parametric surfaces (Sec. 4.4).  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
may import this module; the library never does.

Surfaces are sets of untrimmed bicubic Bezier patches, control points
``C[p][i][j]`` (i along u, j along v, 4 x 4 x 3), S(u, v) = sum B_i(u) B_j(v) C_ij
on [0, 1]^2, oriented by n = S_u x S_v.

* :func:`w_direct` - the plain definition (Eq. 1): w(p) = (1/4pi) times the
  solid angle, the surface integral of (S - p) . (S_u x S_v) / |S - p|^3 over
  every patch, by adaptive 2-D quadrature (scipy's dblquad, a library
  primitive).  Valid away from the surface.
* :func:`boundary_curves` - the oriented boundary of the union: each patch's
  four edge curves counter-clockwise about n (v = 0 along +u, u = 1 along +v,
  v = 1 along -u, u = 0 along -v); a curve and its exact reverse cancel.
* :func:`integrand` / :func:`boundary_term` - Algorithm 2's boundary integrand
  f(phi, t) = (w - d eta) / 4pi with x0 = +z, x1 = -z, written from the
  algorithm's definitions, and its integral by scipy's adaptive quad.

Pins (tests/test_oracle_parametric.py): the rectangle closed form for a flat
patch, w = 1 / 0 inside / outside a cube of six flat patches, boundary
extraction on a grid of patches, and chi + boundary term = w_direct (an
integer chi) for curved patches.
"""
from __future__ import annotations

import math

import numpy as np

X0 = np.array([0.0, 0.0, 1.0])
X1 = -X0


def _bern3(t):
    s = 1.0 - t
    return np.array([s * s * s, 3 * s * s * t, 3 * s * t * t, t * t * t])


def _bern2(t):
    s = 1.0 - t
    return np.array([s * s, 2 * s * t, t * t])


def surface(C, u, v):
    """S, S_u, S_v of one patch at (u, v)."""
    C = np.asarray(C, dtype=np.float64)
    bu, bv = _bern3(u), _bern3(v)
    du, dv = _bern2(u), _bern2(v)
    S = np.einsum("i,j,ijk->k", bu, bv, C)
    Su = 3.0 * np.einsum("i,j,ijk->k", du, bv, C[1:] - C[:-1])
    Sv = 3.0 * np.einsum("i,j,ijk->k", bu, dv, C[:, 1:] - C[:, :-1])
    return S, Su, Sv


def w_direct(patches, p, eps=1e-10):
    """(1/4pi) sum over patches of the solid-angle integral (Eq. 1)."""
    from scipy.integrate import dblquad
    p = np.asarray(p, dtype=np.float64)
    total = 0.0
    for C in np.asarray(patches, dtype=np.float64):
        def f(v, u, C=C):
            S, Su, Sv = surface(C, u, v)
            r = S - p
            n = np.cross(Su, Sv)
            return float(r @ n) / float(r @ r) ** 1.5
        val, _ = dblquad(f, 0.0, 1.0, 0.0, 1.0, epsabs=eps, epsrel=eps)
        total += val
    return total / (4.0 * math.pi)


def patch_edges(C):
    """The four boundary curves of one patch, counter-clockwise about S_u x S_v."""
    C = np.asarray(C, dtype=np.float64)
    return [C[:, 0].copy(), C[3, :].copy(), C[::-1, 3].copy(), C[0, ::-1].copy()]


def boundary_curves(patches):
    """Oriented boundary curves (n, 4, 3) of the union: reversed duplicates cancel."""
    curves = [e for C in np.asarray(patches, dtype=np.float64) for e in patch_edges(C)]
    keys = [tuple(np.asarray(c, dtype=np.float32).ravel()) for c in curves]
    rkeys = [tuple(np.asarray(c[::-1], dtype=np.float32).ravel()) for c in curves]
    count = {}
    for k in keys:
        count[k] = count.get(k, 0) + 1
    out = []
    used = {}
    for c, k, rk in zip(curves, keys, rkeys):
        # net multiplicity of this oriented curve: copies minus reversed copies
        net = count.get(k, 0) - count.get(rk, 0)
        if net > 0 and used.get(k, 0) < net:
            out.append(c)
            used[k] = used.get(k, 0) + 1
    return np.array(out).reshape(-1, 4, 3)


def _curve(P, t):
    P = np.asarray(P, dtype=np.float64)
    b = _bern3(t)
    d = _bern2(t)
    return b @ P, 3.0 * (d @ (P[1:] - P[:-1]))


def integrand(P, p, t):
    """Algorithm 2's f(phi, t) = (w - d eta) / 4pi for the cubic curve P at t."""
    phi, dphi = _curve(P, t)
    r = phi - np.asarray(p, dtype=np.float64)
    L = math.sqrt(float(r @ r))
    G = r / L
    dG = (dphi - (G @ dphi) * G) / L
    X = X0 - (X0 @ G) * G
    dX = -(X0 @ dG) * G - (X0 @ G) * dG
    deta = float(G @ np.cross(X, dX)) / float(X @ X)
    v = G - (X1 @ G) * X1
    dv = dG - (X1 @ dG) * X1
    w = float(X1 @ np.cross(v, dv)) / float(v @ v)
    return (w - deta) / (4.0 * math.pi)


def boundary_term(curves, p, eps=1e-12):
    from scipy.integrate import quad
    total = 0.0
    for P in curves:
        val, _ = quad(lambda t: integrand(P, p, t), 0.0, 1.0, epsabs=eps, epsrel=eps, limit=400)
        total += val
    return total
