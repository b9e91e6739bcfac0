"""Pins of the oracle's solid-angle sums against closed forms (no GPU).

Each test ties ``oracle.direct`` / ``oracle.triangle_area`` / ``oracle.antipodal``
to a value fixed by geometry rather than by re-typing the oracle's own formula:
Girard's theorem with independently computed interior angles (Sec. 3.3, Eq. 5),
the closed-form solid angle of an axis-centred rectangle and of a disk, integer
values for closed meshes (Sec. 3.2), additivity over a split mesh, orientation
reversal, and the unit jump across a face (the Alexander numbering, Sec. 4.2).
"""
import math

import numpy as np
import pytest

import gen
import oracle

FOUR_PI = 4.0 * math.pi


def _girard(A, B, C):
    """Unsigned area of the small spherical triangle via interior angles."""
    def angle(P, Q, R):
        t1 = Q - np.dot(P, Q) * P
        t2 = R - np.dot(P, R) * P
        c = np.dot(t1, t2) / (np.linalg.norm(t1) * np.linalg.norm(t2))
        return math.acos(max(-1.0, min(1.0, c)))
    return angle(A, B, C) + angle(B, C, A) + angle(C, A, B) - math.pi


def test_single_triangle_matches_girard():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(400):
        a, b, c, q = (rng.normal(size=3).astype(np.float32) for _ in range(4))
        u = [(x.astype(np.float64) - q.astype(np.float64)) for x in (a, b, c)]
        u = [x / np.linalg.norm(x) for x in u]
        det = np.dot(u[0], np.cross(u[1], u[2]))
        if abs(det) < 1e-3:
            continue
        area = oracle.triangle_area(a, b, c, q)
        g = _girard(*u)
        assert math.copysign(1.0, area) == math.copysign(1.0, det)
        assert abs(abs(area) - g) < 1e-10, (area, g)
        checked += 1
    assert checked > 300


def _rect_mesh(a, b):
    V = np.array([[-a, -b, 0], [a, -b, 0], [a, b, 0], [-a, b, 0]], dtype=np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return V, F


@pytest.mark.parametrize("a,b,h", [(1.0, 1.0, 1.0), (0.5, 2.0, 0.25), (3.0, 0.125, 2.0)])
def test_rectangle_on_axis(a, b, h):
    # Omega = 4 arcsin(ab / sqrt((a^2+h^2)(b^2+h^2))) for the rectangle
    # [-a,a]x[-b,b] seen from (0,0,-h) (it faces +z, so the viewer is behind it).
    V, F = _rect_mesh(a, b)
    q = np.array([[0.0, 0.0, -h]], dtype=np.float32)
    hq = float(np.float32(h))
    omega = 4.0 * math.asin(a * b / math.sqrt((a * a + hq * hq) * (b * b + hq * hq)))
    w = oracle.direct(V, F, q)[0]
    assert abs(w - omega / FOUR_PI) < 1e-12
    # viewed from the front the sign flips
    w2 = oracle.direct(V, F, -q)[0]
    assert abs(w2 + omega / FOUR_PI) < 1e-12


def _cube():
    V = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], dtype=np.float32)
    quads = []
    # faces as (axis, value) with CCW order seen from outside
    for axis in range(3):
        for s in (-1, 1):
            idx = [i for i in range(8) if V[i, axis] == s]
            P = V[idx].astype(np.float64)
            c = P.mean(0)
            n = np.zeros(3); n[axis] = s
            # order by angle around the face normal
            u = np.zeros(3); u[(axis + 1) % 3] = 1
            v = np.cross(n, u)
            ang = [math.atan2(np.dot(p - c, v), np.dot(p - c, u)) for p in P]
            order = [idx[k] for k in np.argsort(ang)]
            quads.append(order)
    F = []
    for qd in quads:
        F.append([qd[0], qd[1], qd[2]])
        F.append([qd[0], qd[2], qd[3]])
    return V, np.array(F, dtype=np.int32)


def test_cube_face_from_centre_is_one_sixth():
    V, F = _cube()
    q = np.zeros((1, 3), dtype=np.float32)
    for f in range(6):
        w = oracle.direct(V, F[2 * f:2 * f + 2], q)[0]
        assert abs(w - 1.0 / 6.0) < 1e-14
    assert abs(oracle.direct(V, F, q)[0] - 1.0) < 1e-14


def test_closed_icosphere_inside_outside():
    V, F = gen.icosphere(3)
    V = V.astype(np.float32); F = F.astype(np.int32)
    rng = np.random.default_rng(3)
    inner = (rng.normal(size=(200, 3)) * 0.2).astype(np.float32)
    inner = inner[np.linalg.norm(inner, axis=1) < 0.9]
    outer = rng.normal(size=(200, 3))
    outer = (outer / np.linalg.norm(outer, axis=1, keepdims=True) * rng.uniform(1.1, 5, (200, 1))).astype(np.float32)
    assert np.max(np.abs(oracle.direct(V, F, inner) - 1.0)) < 1e-12
    assert np.max(np.abs(oracle.direct(V, F, outer))) < 1e-12


def test_disk_on_axis_matches_cap_formula():
    # Omega = 2 pi (1 - h / sqrt(h^2 + R^2)) for a disk of radius R; a fan of n
    # triangles inscribed in the circle differs by O((pi/n)^2) relative.
    n, R = 4096, 1.0
    t = 2 * np.pi * np.arange(n) / n
    V = np.concatenate([[[0, 0, 0]], np.stack([R * np.cos(t), R * np.sin(t), np.zeros(n)], 1)]).astype(np.float32)
    F = np.stack([np.zeros(n), 1 + np.arange(n), 1 + (np.arange(n) + 1) % n], 1).astype(np.int32)
    for h in (0.1, 0.5, 2.0):
        q = np.array([[0, 0, -h]], dtype=np.float32)
        omega = 2 * math.pi * (1 - h / math.sqrt(h * h + R * R))
        w = oracle.direct(V, F, q)[0]
        assert abs(w * FOUR_PI - omega) / omega < 5 * (math.pi / n) ** 2


def _left_region_area(V, E):
    """Area of the spherical region left of the boundary loop E (geodesic edges,
    seen from the origin) by Gauss-Bonnet (Eq. 7 with k_g = 0):
    2 pi - sum of the signed exterior turning angles at the corners."""
    nxt = {int(a): int(b) for a, b in E}
    start = int(E[0, 0])
    loop = [start]
    while nxt[loop[-1]] != start:
        loop.append(nxt[loop[-1]])
    P = V[loop].astype(np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    n = len(P)
    turning = 0.0
    for i in range(n):
        a, b, c = P[i - 1], P[i], P[(i + 1) % n]
        t_in = -(a - np.dot(b, a) * b)       # direction of travel arriving at b
        t_out = c - np.dot(b, c) * b         # direction of travel leaving b
        turning += math.atan2(np.dot(b, np.cross(t_in, t_out)), np.dot(t_in, t_out))
    return 2.0 * math.pi - turning, len(loop)


def test_open_cap_from_centre_equals_gauss_bonnet():
    m = gen.small_cap(3, 0.8)
    E = oracle.boundary(m.F, m.nv)
    area, nloop = _left_region_area(m.V, E)
    assert nloop == len(E) == 36
    w = oracle.direct(m.V, m.F, np.zeros((1, 3), np.float32))[0]
    assert abs(w - area / FOUR_PI) < 1e-12


def test_additivity_cap_plus_complement():
    V, F = gen.icosphere(3)
    V = V.astype(np.float32); F = F.astype(np.int32)
    cz = V[F].astype(np.float64).mean(1)[:, 2]
    cap, rest = F[cz <= 0.8], F[cz > 0.8]
    Q = gen.workload("small")[1][:300]
    wc = oracle.direct(V, cap, Q)
    wr = oracle.direct(V, rest, Q)
    wall = oracle.direct(V, F, Q)
    assert np.max(np.abs(wc + wr - wall)) < 1e-12
    assert np.max(np.abs(wall - np.round(wall))) < 1e-12


def test_orientation_reversal_negates():
    m, Q = gen.workload("small", n_query=300)
    w = oracle.direct(m.V, m.F, Q)
    wr = oracle.direct(m.V, m.F[:, ::-1].copy(), Q)
    assert np.max(np.abs(w + wr)) < 1e-13


def test_unit_jump_across_face():
    # crossing a face along its normal lowers w by exactly one
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float32)
    F = np.array([[0, 1, 2]], dtype=np.int32)
    dev = []
    for d in (1e-2, 1e-3, 1e-4, 1e-5):
        q = np.array([[0.25, 0.25, -d], [0.25, 0.25, d]], dtype=np.float32)
        w = oracle.direct(V, F, q)
        assert w[0] > 0 > w[1]
        dev.append(abs((w[1] - w[0]) + 1.0))
    # the deviation from -1 vanishes linearly with the distance to the face
    for k in range(3):
        assert dev[k + 1] < dev[k] / 5.0
    assert dev[-1] < 1e-4


def test_far_field_decays():
    m, _ = gen.workload("small", n_query=1)
    far = np.array([[1e3, 0, 0], [0, 1e4, 0], [0, 0, -1e5]], dtype=np.float32)
    w = oracle.direct(m.V, m.F, far)
    assert np.all(np.abs(w) < 1e-4)
