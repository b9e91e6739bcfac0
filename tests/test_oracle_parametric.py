"""Pins of oracle/parametric.py (Sec. 4.4) to facts other than itself.

* A flat patch (a bilinear map written as a bicubic patch) over the rectangle
  [-a, a] x [-b, b] seen from (0, 0, h): w = -Omega / 4pi with the closed-form
  solid angle Omega = 4 arcsin(ab / sqrt((a^2 + h^2)(b^2 + h^2))).
* Six flat patches with outward normals close a cube: w = 1 inside, 0 outside,
  and every edge curve cancels against its neighbour's.
* A 2 x 2 grid of patches keeps only its 8 outer edge curves.
* Algorithm 2's boundary integrand against the definition: for curved patches,
  w_direct - (boundary term) is an integer (the crossing count) at every
  query away from the surface.
"""
import math

import numpy as np
import pytest

pytest.importorskip("scipy")

from oracle import parametric as par  # noqa: E402


def flat_patch(p00, p10, p01, p11):
    """Bicubic control net of the bilinear map through the four corners."""
    C = np.zeros((4, 4, 3))
    for i in range(4):
        for j in range(4):
            u, v = i / 3.0, j / 3.0
            C[i, j] = ((1 - u) * (1 - v) * np.asarray(p00) + u * (1 - v) * np.asarray(p10)
                       + (1 - u) * v * np.asarray(p01) + u * v * np.asarray(p11))
    return C


def cube(s=1.5):
    x, y, z = np.eye(3) * s
    c = lambda *v: np.asarray(v, dtype=np.float64)  # noqa: E731
    faces = [  # (origin corner, u direction, v direction) with u x v outward
        (c(-s, -s, s), 2 * x, 2 * y),      # +z
        (c(-s, -s, -s), 2 * y, 2 * x),     # -z
        (c(s, -s, -s), 2 * y, 2 * z),      # +x
        (c(-s, -s, -s), 2 * z, 2 * y),     # -x
        (c(-s, s, -s), 2 * z, 2 * x),      # +y
        (c(-s, -s, -s), 2 * x, 2 * z),     # -y
    ]
    return np.array([flat_patch(o, o + du, o + dv, o + du + dv) for o, du, dv in faces])


@pytest.mark.parametrize("a,b,h", [(1.0, 1.0, 1.0), (0.5, 2.0, 0.25), (1.5, 0.75, -2.0)])
def test_flat_rectangle_closed_form(a, b, h):
    P = flat_patch([-a, -b, 0], [a, -b, 0], [-a, b, 0], [a, b, 0])
    w = par.w_direct([P], [0.0, 0.0, h])
    omega = 4.0 * math.asin(a * b / math.sqrt((a * a + h * h) * (b * b + h * h)))
    assert abs(w - (-math.copysign(omega, h) / (4 * math.pi))) < 1e-8


def test_cube_inside_outside_and_cancelled_edges():
    C = cube()
    assert par.boundary_curves(C).shape[0] == 0
    for p, want in (([0.1, -0.2, 0.3], 1.0), ([2.5, 0.0, 0.1], 0.0), ([0.0, 0.0, -3.0], 0.0)):
        assert abs(par.w_direct(C, p) - want) < 1e-8


def test_grid_keeps_outer_edges():
    P = [flat_patch([i, j, 0], [i + 1, j, 0], [i, j + 1, 0], [i + 1, j + 1, 0]) for i in range(2) for j in range(2)]
    E = par.boundary_curves(P)
    assert E.shape == (8, 4, 3)
    # every outer curve runs counter-clockwise about +z: its start is its predecessor's end
    ends = {tuple(e[3]) for e in E}
    assert all(tuple(e[0]) in ends for e in E)


def _wavy_patch(rng, z0=0.0):
    C = flat_patch([-1, -1, z0], [1, -1, z0], [-1, 1, z0], [1, 1, z0])
    C[:, :, 2] += rng.uniform(-0.4, 0.4, size=(4, 4))
    return C


def test_algorithm2_integrand_against_definition():
    rng = np.random.default_rng(3)
    patches = [_wavy_patch(rng)]
    curves = par.boundary_curves(patches)
    assert curves.shape[0] == 4
    for p in rng.uniform(-1.5, 1.5, size=(12, 3)):
        wd = par.w_direct(patches, p)
        bt = par.boundary_term(curves, p)
        chi = wd - bt
        assert abs(chi - round(chi)) < 1e-7, (p, wd, bt)
