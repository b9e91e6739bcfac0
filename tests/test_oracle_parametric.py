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
* The patch evaluation itself: an affine control net reproduces the affine
  map (linear precision of the Bernstein basis); the net with z coefficients
  c_i d_j, c = (0, 0, 1/3, 1) (u^2) and d = (0, 0, 0, 1) (v^3), reproduces
  z = u^2 v^3 and its derivatives (a transposed index gives v^2 u^3); the
  corners interpolate; S_u, S_v match central differences of S.
* The patch's edge curves: as cubic Bezier curves they trace S(t, 0), S(1, t),
  S(1 - t, 1), S(0, 1 - t), close into one loop, and on a flat patch enclose
  its area with the sign of the normal (shoelace).
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


@pytest.mark.parametrize("a,b,h", [(1.0, 1.0, 1.0), (0.5, 2.0, 0.25), (1.5, 0.75, -2.0)])
def test_w_gauss_rectangle_closed_form(a, b, h):
    P = flat_patch([-a, -b, 0], [a, -b, 0], [-a, b, 0], [a, b, 0])
    w = par.w_gauss([P], [0.0, 0.0, h])
    omega = 4.0 * math.asin(a * b / math.sqrt((a * a + h * h) * (b * b + h * h)))
    assert abs(w - (-math.copysign(omega, h) / (4 * math.pi))) < 1e-6


def test_w_gauss_cube():
    C = cube()
    for p, want in (([0.1, -0.2, 0.3], 1.0), ([2.5, 0.0, 0.1], 0.0), ([0.0, 0.0, -3.0], 0.0)):
        assert abs(par.w_gauss(C, p) - want) < 1e-6


def test_w_gauss_matches_definition_on_curved_patches():
    rng = np.random.default_rng(11)
    patches = [_wavy_patch(rng), _wavy_patch(rng, z0=0.3)]
    for p in ([0.2, -0.1, 1.2], [-0.6, 0.4, -0.9], [1.4, 1.3, 0.2]):
        assert abs(par.w_gauss(patches, p) - par.w_direct(patches, p, eps=1e-9)) < 1e-5


def test_integrand_is_the_monopole_potential():
    """f dt = -(1 + cos theta) d(azimuth) / 4pi about q with the pole along x0 = +z:
    theta and the azimuth from the spherical angles of phi(t) - q, the azimuth's
    rate by central differences of its unwrapped value."""
    rng = np.random.default_rng(5)
    for _ in range(6):
        P = rng.uniform(-1, 1, size=(4, 3))
        q = rng.uniform(-0.5, 0.5, size=3)
        for t in (0.1, 0.37, 0.5, 0.81):
            h = 1e-6
            az = []
            for s in (t - h, t, t + h):
                phi = _bern(s) @ P
                r = phi - q
                az.append(math.atan2(r[1], r[0]))
            az = np.unwrap(az)
            daz = (az[2] - az[0]) / (2 * h)
            r = _bern(t) @ P - q
            cos_t = r[2] / np.linalg.norm(r)
            want = -(1.0 + cos_t) * daz / (4 * math.pi)
            got = par.integrand(P, q, t)
            assert abs(got - want) <= 1e-6 * (1.0 + abs(want)), (t, got, want)


def _bern(t):
    s = 1.0 - t
    return np.array([s ** 3, 3 * s * s * t, 3 * s * t * t, t ** 3])


def test_boundary_scale_bounds_the_term():
    from scipy.integrate import quad
    rng = np.random.default_rng(8)
    patches = [_wavy_patch(rng)]
    curves = par.boundary_curves(patches)
    for p in rng.uniform(-1.5, 1.5, size=(4, 3)):
        labs = sum(quad(lambda t: abs(par.integrand(P, p, t)), 0, 1, limit=400)[0] for P in curves)
        assert par.boundary_scale(curves, p) >= labs * (1 - 1e-6) - 1e-9
        assert labs >= abs(par.boundary_term(curves, p)) - 1e-9
    # a circle-like loop about the z axis above a query on the axis, traversed
    # once: in every quadrant r_x r'_y >= 0 >= r_y r'_x, so the scale equals
    # |f|'s integral, and f keeps one sign, so that equals |boundary term|
    k = 4.0 * (math.sqrt(2.0) - 1.0) / 3.0
    quarter = lambda a0: np.array([[math.cos(a0), math.sin(a0), 1.0],  # noqa: E731
                                   [math.cos(a0) - k * math.sin(a0), math.sin(a0) + k * math.cos(a0), 1.0],
                                   [math.cos(a0 + math.pi / 2) + k * math.sin(a0 + math.pi / 2),
                                    math.sin(a0 + math.pi / 2) - k * math.cos(a0 + math.pi / 2), 1.0],
                                   [math.cos(a0 + math.pi / 2), math.sin(a0 + math.pi / 2), 1.0]])
    loop = np.array([quarter(j * math.pi / 2) for j in range(4)])
    p = [0.0, 0.0, 0.0]
    bt, ba = par.boundary_term(loop, p), par.boundary_scale(loop, p)
    assert bt < 0 and abs(ba + bt) <= 1e-7 * ba


def test_inconsistent_orientation_keeps_the_shared_edge_twice():
    """Two patches on either side of the edge x = 1 with opposite normals (the
    second one flipped): both traverse the shared edge in the same direction,
    so it does not cancel but has net multiplicity 2 (the surface boundary
    read as a 1-chain)."""
    A = flat_patch([0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0])          # u along +x: edge u = 1 runs +y
    B = flat_patch([2, 1, 0], [1, 1, 0], [2, 0, 0], [1, 0, 0])          # u along -x: edge u = 1 runs -y ...
    B = B[:, ::-1].copy()                                              # ... flipped in v: now +y, like A's
    E = par.boundary_curves([A, B])
    shared = [e for e in E if np.allclose(e[:, 0], 1.0)]
    assert len(shared) == 2 and all(e[3, 1] > e[0, 1] for e in shared)


def test_degenerate_patch_has_no_boundary():
    C = np.ones((4, 4, 3)) * 0.25
    assert par.boundary_curves([C]).shape[0] == 0
    assert abs(par.w_gauss([C], [0.0, 0.0, 1.0])) < 1e-15


def test_integrand_continuous_through_the_antipode():
    """Where the curve passes exactly along x1 = -z from the query, Algorithm 2's
    w and d eta are each undefined but their difference is continuous (the
    monopole form -(1 + cos theta) d(azimuth) / 4pi vanishes as theta -> pi): the
    oracle's value there (0) is the limit of its values at nearby queries."""
    P = np.array([[1.0, 0.0, 0.0], [1.0, 1 / 3, 0.0], [1.0, 2 / 3, 0.0], [1.0, 1.0, 0.0]])
    assert par.integrand(P, [1.0, 0.5, 0.8], 0.5) == 0.0
    vals = [abs(par.integrand(P, [1.0 + e, 0.5, 0.8], 0.5)) for e in (1e-2, 1e-3, 1e-4)]
    assert vals[0] > vals[1] > vals[2] and vals[2] < 1e-3


def test_surface_linear_precision_and_corners():
    rng = np.random.default_rng(3)
    a0, a1, a2 = rng.normal(size=(3, 3))
    C = np.array([[a0 + a1 * (i / 3.0) + a2 * (j / 3.0) for j in range(4)] for i in range(4)])
    for u, v in rng.uniform(0, 1, size=(10, 2)):
        S, Su, Sv = par.surface(C, u, v)
        assert np.allclose(S, a0 + a1 * u + a2 * v, atol=1e-14)
        assert np.allclose(Su, a1, atol=1e-13) and np.allclose(Sv, a2, atol=1e-13)
    C = rng.normal(size=(4, 4, 3))
    for (u, v), (i, j) in (((0, 0), (0, 0)), ((1, 0), (3, 0)), ((0, 1), (0, 3)), ((1, 1), (3, 3))):
        assert np.allclose(par.surface(C, u, v)[0], C[i, j], atol=1e-15)


def test_surface_reproduces_u2_v3():
    c = np.array([0.0, 0.0, 1.0 / 3.0, 1.0])     # Bernstein coefficients of u^2
    d = np.array([0.0, 0.0, 0.0, 1.0])           # of v^3
    C = np.zeros((4, 4, 3))
    C[:, :, 2] = np.outer(c, d)
    for u, v in ((0.3, 0.7), (0.9, 0.2), (0.5, 0.5)):
        S, Su, Sv = par.surface(C, u, v)
        assert abs(S[2] - u * u * v ** 3) < 1e-15
        assert abs(Su[2] - 2 * u * v ** 3) < 1e-14
        assert abs(Sv[2] - 3 * u * u * v * v) < 1e-14


def test_surface_derivatives_against_differences():
    rng = np.random.default_rng(4)
    C = rng.normal(size=(4, 4, 3))
    h = 1e-6
    for u, v in rng.uniform(0.1, 0.9, size=(6, 2)):
        _, Su, Sv = par.surface(C, u, v)
        fu = (par.surface(C, u + h, v)[0] - par.surface(C, u - h, v)[0]) / (2 * h)
        fv = (par.surface(C, u, v + h)[0] - par.surface(C, u, v - h)[0]) / (2 * h)
        assert np.allclose(Su, fu, atol=1e-8) and np.allclose(Sv, fv, atol=1e-8)


def test_patch_edges_trace_the_boundary_counter_clockwise():
    rng = np.random.default_rng(5)
    C = rng.normal(size=(4, 4, 3))
    e = par.patch_edges(C)
    params = [lambda t: (t, 0.0), lambda t: (1.0, t), lambda t: (1.0 - t, 1.0), lambda t: (0.0, 1.0 - t)]
    for k in range(4):
        assert np.allclose(e[k][3], e[(k + 1) % 4][0], atol=0)          # one closed loop
        for t in (0.0, 0.25, 0.6, 1.0):
            want = par.surface(C, *params[k](t))[0]
            got = par._curve(e[k], t)[0]
            assert np.allclose(got, want, atol=1e-14)
    # flat patch over [0, 2] x [0, 1]: the loop encloses area 2, counter-clockwise about +z
    F = flat_patch((0, 0, 0), (2, 0, 0), (0, 1, 0), (2, 1, 0))
    assert np.allclose(np.cross(*par.surface(F, 0.5, 0.5)[1:]), [0, 0, 2])
    pts = np.concatenate([[par._curve(c, t)[0] for t in np.linspace(0, 1, 9)[:-1]] for c in par.patch_edges(F)])
    x, y = pts[:, 0], pts[:, 1]
    assert abs(0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) - 2.0) < 1e-12
    # the same patch with u and v swapped has normal -z and a clockwise loop
    pts = np.concatenate([[par._curve(c, t)[0] for t in np.linspace(0, 1, 9)[:-1]]
                          for c in par.patch_edges(F.transpose(1, 0, 2))])
    x, y = pts[:, 0], pts[:, 1]
    assert abs(0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) + 2.0) < 1e-12
