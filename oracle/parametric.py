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
* :func:`boundary_scale` - the integral over the curves of
  (|r_x r'_y| + |r_y r'_x|) (1 + cos theta) / (4pi rho^2), r = phi - p,
  rho^2 = r_x^2 + r_y^2: f is minus the same expression without the absolute
  values (the monopole form), so this bounds the integral of |f| and sets the
  scale of the rounding error of an evaluation of f from r and r'.
* :func:`w_gauss` - the definition (Eq. 1) by a fixed tensor Gauss-Legendre
  rule on a uniform split of each patch (numpy's leggauss), vectorised: far
  faster than :func:`w_direct`, accurate for queries a few sub-patch widths
  from the surface; used to fix the integer crossing count of such queries.

Pins (tests/test_oracle_parametric.py): the rectangle closed form for a flat
patch, w = 1 / 0 inside / outside a cube of six flat patches (both for
w_direct and w_gauss), boundary extraction on a grid of patches, chi +
boundary term = w_direct (an integer chi) for curved patches, and the
integrand against the monopole form -(1 + cos theta) d(azimuth) / 4pi
computed from spherical angles; the patch evaluation by linear precision,
reproduction of u^2 v^3, corner interpolation and central differences; the
edge curves by tracing the patch boundary as one counter-clockwise loop.
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
    if float(X @ X) == 0.0 and G[2] < 0.0:
        # the curve point lies exactly along x1 from p: w and d eta are each
        # undefined there, their difference tends to 0 (a removable point)
        return 0.0
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


def boundary_scale(curves, p, eps=1e-8):
    """Sum over the curves of the integral of (|r_x r'_y| + |r_y r'_x|) (1 + cos theta)
    / (4pi rho^2) (scipy's adaptive quad)."""
    from scipy.integrate import quad
    p = np.asarray(p, dtype=np.float64)

    def g(P, t):
        phi, dphi = _curve(P, t)
        r = phi - p
        rho2 = r[0] * r[0] + r[1] * r[1]
        if rho2 == 0.0:
            return 0.0
        cos_t = r[2] / math.sqrt(float(r @ r))
        return (abs(r[0] * dphi[1]) + abs(r[1] * dphi[0])) * (1.0 + cos_t) / (4.0 * math.pi * rho2)

    total = 0.0
    for P in curves:
        val, _ = quad(lambda t: g(P, t), 0.0, 1.0, epsabs=eps, epsrel=1e-6, limit=400)
        total += val
    return total


def w_gauss(patches, p, n_sub=8, order=8):
    """(1/4pi) times the solid angle (Eq. 1), each patch split into n_sub x n_sub
    parameter squares, each integrated by the order x order Gauss-Legendre rule."""
    x, wts = np.polynomial.legendre.leggauss(order)
    edges = np.arange(n_sub) / n_sub
    nodes = (edges[:, None] + (x[None, :] + 1.0) / (2 * n_sub)).ravel()          # [n_sub * order]
    weights = np.tile(wts / (2 * n_sub), n_sub)
    bu = np.stack([_bern3(t) for t in nodes])                                       # [m, 4]
    du = np.stack([_bern2(t) for t in nodes])                                       # [m, 3]
    p = np.asarray(p, dtype=np.float64)
    total = 0.0
    for C in np.asarray(patches, dtype=np.float64):
        S = np.einsum("ai,bj,ijk->abk", bu, bu, C)
        Su = 3.0 * np.einsum("ai,bj,ijk->abk", du, bu, C[1:] - C[:-1])
        Sv = 3.0 * np.einsum("ai,bj,ijk->abk", bu, du, C[:, 1:] - C[:, :-1])
        r = S - p
        n = np.cross(Su, Sv)
        f = np.einsum("abk,abk->ab", r, n) / np.einsum("abk,abk->ab", r, r) ** 1.5
        total += float(weights @ f @ weights)
    return total / (4.0 * math.pi)
