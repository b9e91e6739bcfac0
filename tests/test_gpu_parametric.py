"""Parametric surfaces on the GPU (Sec. 4.4, Algorithm 2) against oracle/parametric.py.

w against the plain definition (the surface solid-angle integral, adaptive 2-D
quadrature, or its fixed Gauss rule for the 100-patch workload); chi against
the integer w_direct - (boundary term of the oracle's own Algorithm 2
integrand); boundary extraction against the oracle's.  Queries stay at least
0.02 from the surface (the crossing count is only defined off the surface,
and a query within the bilinear tolerance may be counted either way).

Tolerances on w:
* fp64 = 1: each curve's integral to quad_tol = 1e-10 per unit of parameter
  (nc * 1e-10 in all), the oracle's to 1e-12, plus the FP32 output rounding:
  1e-7 covers it.
* fp64 = 0 (FP32 panels): in addition each panel may stop at 2^-20 of its own
  rounding scale (only while that is below 2^-18 / 4pi in absolute terms),
  and its 15 FP32 values carry a few units of rounding of the same scale:
  nc * quad_tol + 2^-19 * S + 2^-24 (|w| + 1), S the oracle's boundary_scale.
  On the 100-patch workload FP32 and FP64 panels are also compared on every
  cell against 1e-5 (the cap keeps near-string panels out of FP32).
"""
import math

import numpy as np
import pytest

pytest.importorskip("scipy")
torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import parametric as par  # noqa: E402

QUAD_TOL = 1e-10
TOL_W64 = 1e-7


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


def flat_patch(p00, p10, p01, p11):
    C = np.zeros((4, 4, 3))
    for i in range(4):
        for j in range(4):
            u, v = i / 3.0, j / 3.0
            C[i, j] = ((1 - u) * (1 - v) * np.asarray(p00, float) + u * (1 - v) * np.asarray(p10, float)
                       + (1 - u) * v * np.asarray(p01, float) + u * v * np.asarray(p11, float))
    return C


def wavy_grid(rng, n=2, amp=0.35):
    """n x n patches over [-1, 1]^2 sharing their edge control points, random heights."""
    g = 3 * n + 1
    xs = np.linspace(-1.0, 1.0, g)
    Z = rng.uniform(-amp, amp, size=(g, g))
    P = []
    for a in range(n):
        for b in range(n):
            C = np.zeros((4, 4, 3))
            for i in range(4):
                for j in range(4):
                    C[i, j] = [xs[3 * a + i], xs[3 * b + j], Z[3 * a + i, 3 * b + j]]
            P.append(C)
    return np.array(P, dtype=np.float32).astype(np.float64)


def surface_samples(patches, res=120):
    grid = np.linspace(0, 1, res)
    return np.concatenate([np.array([par.surface(C, u, v)[0] for u in grid for v in grid]) for C in patches])


def far_queries(patches, rng, n, lo=-1.4, hi=1.4, margin=0.02):
    pts = []
    samples = surface_samples(patches)
    while len(pts) < n:
        q = rng.uniform(lo, hi, size=3)
        if np.min(np.linalg.norm(samples - q, axis=1)) > margin:
            pts.append(q)
    return np.array(pts, dtype=np.float32)


def tol_w(fp64, curves, q, w):
    nc = len(curves)
    if fp64:
        return TOL_W64 + nc * QUAD_TOL
    return nc * QUAD_TOL + 2.0 ** -19 * par.boundary_scale(curves, q) + 2.0 ** -24 * (abs(w) + 1.0)


def _check(gwn, patches, Q, fp64):
    curves = par.boundary_curves(patches)
    with gwn.ParamSurface(np.asarray(patches, np.float32), fp64=fp64, quad_tol=QUAD_TOL) as s:
        E = s.boundary_curves()
        assert E.shape == curves.shape and np.array_equal(E, curves.astype(np.float32))
        w, chi = s.query(torch.from_numpy(Q).cuda())
        st = s.status()
    w = w.cpu().numpy().astype(np.float64)
    chi = chi.cpu().numpy()
    assert st["budget_hits"] == 0 and st["unconverged"] == 0, st
    for k, q in enumerate(Q.astype(np.float64)):
        wd = par.w_direct(patches, q)
        assert abs(w[k] - wd) <= tol_w(fp64, curves, q, wd), (q, w[k], wd)
        bt = par.boundary_term(curves, q)
        assert chi[k] == round(wd - bt), (q, chi[k], wd - bt)
    return w, chi


@pytest.mark.parametrize("fp64", [0, 1])
def test_flat_rectangle(gwn, fp64):
    P = np.array([flat_patch([-1, -0.5, 0], [1, -0.5, 0], [-1, 0.5, 0], [1, 0.5, 0])])
    Q = np.array([[0, 0, 1.0], [0, 0, -0.5], [0.3, -0.2, 0.25], [2.0, 0.0, 0.1]], np.float32)
    w, chi = _check(gwn, P, Q, fp64)
    h = 1.0
    omega = 4.0 * math.asin(1.0 * 0.5 / math.sqrt((1 + h * h) * (0.25 + h * h)))
    assert abs(w[0] + omega / (4 * math.pi)) <= 2e-7
    assert np.array_equal(chi, [0, 1, 0, 0])


@pytest.mark.parametrize("fp64", [0, 1])
def test_closed_cube(gwn, fp64):
    s = 1.5
    x, y, z = np.eye(3) * s
    o = lambda *v: np.asarray(v, float)  # noqa: E731
    faces = [(o(-s, -s, s), 2 * x, 2 * y), (o(-s, -s, -s), 2 * y, 2 * x), (o(s, -s, -s), 2 * y, 2 * z),
             (o(-s, -s, -s), 2 * z, 2 * y), (o(-s, s, -s), 2 * z, 2 * x), (o(-s, -s, -s), 2 * x, 2 * z)]
    P = np.array([flat_patch(a, a + du, a + dv, a + du + dv) for a, du, dv in faces])
    Q = np.array([[0.1, -0.2, 0.3], [1.0, 1.0, -1.0], [2.5, 0.0, 0.1], [0.0, 0.0, -3.0], [0.2, 0.3, 2.0]],
                 np.float32)
    with gwn.ParamSurface(P.astype(np.float32), fp64=fp64) as sf:
        assert sf.boundary_curves().shape[0] == 0
        w, chi = sf.query(torch.from_numpy(Q).cuda())
    assert np.array_equal(w.cpu().numpy(), np.array([1, 1, 0, 0, 0], np.float32))


@pytest.mark.parametrize("fp64", [0, 1])
@pytest.mark.parametrize("seed", [1, 2])
def test_curved_patch_grid(gwn, seed, fp64):
    rng = np.random.default_rng(seed)
    P = wavy_grid(rng)
    Q = far_queries(P, rng, 14)
    # rays through the seams x = 0 and y = 0 shared by the 2 x 2 patches, and
    # through their common corner: each crossing is counted once
    seams = np.array([[0, 0, -1.3], [0, 0.41, -1.2], [-0.63, 0, -1.1], [0, -0.27, 1.3], [0, 0, 1.2]],
                     np.float32)
    w, chi = _check(gwn, P, np.concatenate([Q, seams]), fp64)
    assert np.any(chi != 0)      # some rays do cross the surface
    assert np.all(chi[len(Q):] == [1, 1, 1, 0, 0])


def test_empty_inputs(gwn):
    rng = np.random.default_rng(4)
    P = wavy_grid(rng)
    with gwn.ParamSurface(P.astype(np.float32)) as s:
        w, chi = s.query(torch.zeros((0, 3), dtype=torch.float32, device="cuda"))
        assert w.numel() == 0 and chi.numel() == 0
        w, chi = s.query_grid(np.zeros(0, np.float32), np.zeros(3, np.float32), np.zeros(2, np.float32))
        assert w.shape == (2, 3, 0)
    with gwn.ParamSurface(np.zeros((0, 4, 4, 3), np.float32)) as s:
        assert s.boundary_curves().shape == (0, 4, 3)
        w, chi = s.query(torch.ones((3, 3), dtype=torch.float32, device="cuda"))
        assert np.all(w.cpu().numpy() == 0) and np.all(chi.cpu().numpy() == 0)


def _cells(x, y, z):
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)


def _surface_distance(patches, pts, res=60):
    from scipy.spatial import cKDTree
    return cKDTree(surface_samples(patches, res)).query(pts.astype(np.float64))[0]


@pytest.mark.parametrize("fp64", [0, 1])
def test_grid_matches_points(gwn, fp64):
    """Ray reuse per (x, y) column against one ray per cell, on a ragged grid:
    identical chi off the surface, and w from the same boundary code (equal up
    to the order in which a warp's lanes happen to sum their panels)."""
    rng = np.random.default_rng(9)
    P = wavy_grid(rng, n=3)
    x = np.sort(rng.uniform(-1.2, 1.2, 13)).astype(np.float32)
    y = np.sort(rng.uniform(-1.2, 1.2, 10)).astype(np.float32)
    z = np.sort(rng.uniform(-0.8, 0.8, 37)).astype(np.float32)
    cells = _cells(x, y, z)
    with gwn.ParamSurface(P.astype(np.float32), fp64=fp64) as s:
        wg, cg = s.query_grid(x, y, z)
        wp, cp = s.query(torch.from_numpy(cells).cuda())
        st = s.status()
    assert st["budget_hits"] == 0 and st["unconverged"] == 0, st
    far = _surface_distance(P, cells) > 1e-3
    assert far.sum() > 0.9 * len(cells)
    cg, cp = cg.cpu().numpy().ravel(), cp.cpu().numpy()
    assert np.array_equal(cg[far], cp[far])
    assert np.allclose(wg.cpu().numpy().ravel()[far], wp.cpu().numpy()[far], rtol=0, atol=2e-7)
    assert len(set(cg[far].tolist())) >= 2


def test_random_patches_workload(gwn):
    """The 100-random-patch voxel workload (32^3 cells), as the benchmark runs it
    (grid call, FP32 panels): sampled cells against the oracle (chi from the
    fixed Gauss rule of the definition, w = chi + boundary term), FP64 panels
    on the same cells, and ray reuse against one ray per cell everywhere off
    the surface."""
    import gen
    P, Q = gen.param_workload()
    Pd = P.astype(np.float64)
    res = 32
    axes = [np.unique(Q[:, d]) for d in range(3)]
    assert all(len(a) == res for a in axes)
    with gwn.ParamSurface(P) as s:
        wg, cg = s.query_grid(*axes)
        st = s.status(reset=True)
        wp, cp = s.query(torch.from_numpy(Q).cuda())
    with gwn.ParamSurface(P, fp64=1) as s64:
        w64, c64 = s64.query_grid(*axes)
        st64 = s64.status()
    assert st["budget_hits"] == 0 and st["unconverged"] == 0, st
    assert st64["budget_hits"] == 0 and st64["unconverged"] == 0, st64
    wg, cg = wg.cpu().numpy().ravel(), cg.cpu().numpy().ravel()
    dist = _surface_distance(Pd, Q, res=40)
    far = dist > 2e-3
    assert np.array_equal(cg[far], cp.cpu().numpy()[far])
    assert np.array_equal(cg, c64.cpu().numpy().ravel())
    # FP32 against FP64 panels on every cell (FP64 panels meet quad_tol per
    # curve): with the cap on the FP32 rounding level no panel near the ray's
    # string is accepted in FP32 at a large absolute error
    d32 = np.abs(wg - w64.cpu().numpy().ravel())
    print(f"max |w_fp32 - w_fp64| over {len(d32)} cells: {d32.max():.3e}, rms {np.sqrt(np.mean(d32 ** 2)):.3e}")
    assert d32.max() <= 1e-5
    curves = par.boundary_curves(Pd)
    assert len(curves) == 400
    rng = np.random.default_rng(12)
    for k in rng.choice(np.flatnonzero(dist > 0.06), 3, replace=False):
        q = Q[k].astype(np.float64)
        bt = par.boundary_term(curves, q, eps=1e-11)
        chi = round(par.w_gauss(Pd, q, n_sub=16) - bt)
        want = chi + bt
        assert cg[k] == chi, (q, cg[k], chi)
        assert abs(w64.cpu().numpy().ravel()[k] - want) <= TOL_W64 + len(curves) * QUAD_TOL, (q, want)
        assert abs(wg[k] - want) <= tol_w(0, curves, q, want), (q, wg[k], want)


def test_invalid_inputs(gwn):
    """Invalid arguments come back as error statuses; nothing is launched."""
    import ctypes
    rng = np.random.default_rng(5)
    P = wavy_grid(rng).astype(np.float32)
    bad = P.copy()
    bad[0, 1, 2, 0] = np.nan
    with pytest.raises(gwn.GwnError):
        gwn.ParamSurface(bad)
    with pytest.raises(gwn.GwnError):
        gwn.ParamSurface(P, quad_tol=0.0)
    with pytest.raises(gwn.GwnError):
        gwn.ParamSurface(P, max_panels=0)
    lib = gwn.load()
    h = ctypes.c_void_p()
    assert lib.gwn_param_create(P.ctypes.data_as(ctypes.c_void_p), -1, None, ctypes.byref(h)) != 0
    with gwn.ParamSurface(P) as s:
        # z must be non-decreasing
        with pytest.raises(gwn.GwnError):
            s.query_grid(np.zeros(2, np.float32), np.zeros(2, np.float32), np.array([0.5, 0.1], np.float32))
        # queries and outputs must be device memory
        qh = np.zeros((4, 3), np.float32)
        wd = torch.empty(4, dtype=torch.float32, device="cuda")
        rc = lib.gwn_param_query(s._h, qh.ctypes.data_as(ctypes.c_void_p), 4, ctypes.c_void_p(wd.data_ptr()), None,
                                 None)
        assert rc != 0
        with pytest.raises(ValueError):
            s.query(qh)
        assert s.status()["budget_hits"] == 0


def test_inconsistent_orientation_boundary(gwn):
    """Patches on either side of x = 1 with opposite normals: the shared edge is
    kept twice, as in the oracle, and w still matches the definition."""
    A = flat_patch([0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0])
    B = flat_patch([2, 1, 0], [1, 1, 0], [2, 0, 0], [1, 0, 0])[:, ::-1].copy()
    P = np.array([A, B])
    Q = np.array([[0.4, 0.3, 0.5], [1.6, 0.7, -0.5], [1.05, 0.5, 0.8]], np.float32)
    w, chi = _check(gwn, P, Q, 0)
    curves = par.boundary_curves(P)
    assert sum(np.allclose(e[:, 0], 1.0) for e in curves) == 2


def test_grid_axes_in_device_memory(gwn):
    """gwn_param_query_grid with x, y, z in device memory (copied on the stream)
    gives the same cells as with host axes."""
    import ctypes
    rng = np.random.default_rng(13)
    P = wavy_grid(rng).astype(np.float32)
    x = np.sort(rng.uniform(-1.2, 1.2, 7)).astype(np.float32)
    y = np.sort(rng.uniform(-1.2, 1.2, 5)).astype(np.float32)
    z = np.sort(rng.uniform(-0.8, 0.8, 9)).astype(np.float32)
    lib = gwn.load()
    with gwn.ParamSurface(P) as s:
        wh, ch = s.query_grid(x, y, z)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        wd = torch.empty_like(wh)
        cd = torch.empty_like(ch)
        rc = lib.gwn_param_query_grid(s._h, ctypes.c_void_p(dx.data_ptr()), len(x), ctypes.c_void_p(dy.data_ptr()),
                                      len(y), ctypes.c_void_p(dz.data_ptr()), len(z), ctypes.c_void_p(wd.data_ptr()),
                                      ctypes.c_void_p(cd.data_ptr()), None)
        assert rc == 0
        torch.cuda.synchronize()
    assert torch.equal(ch, cd)
    assert np.allclose(wh.cpu().numpy(), wd.cpu().numpy(), rtol=0, atol=2e-7)
