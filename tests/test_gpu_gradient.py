"""GPU gradient of w (Supp. S4, Algorithm 3) against the FP64 oracle.

Tolerance per query and component, derived from the FP32 arithmetic of one
edge term: r, l, v and h carry a few units of rounding u = 2^-24; n and d then
carry absolute errors of order 36 u l0 l1, so c_n = 2 d / (n^2 + d^2) and
c_d = -2 n / (n^2 + d^2) carry a relative error of order 108 u / rho, with
rho = sqrt(n^2 + d^2) / (l0 l1) the unit-vector modulus of the edge's VOS pair;
g_n and g_d add about 20 u.  FP32 partial sums over 64 edges add at most 64 u
of the absolute terms.  Hence
    |grad_gpu - grad_oracle| <= u (128 sum_e |T_e| / rho_e + 128 sum_e |T_e|),
both sums (divided by 4 pi) returned by the oracle.  Queries on the boundary
curve (oracle flag) are excluded: the gradient is undefined there.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


def _check(gwn_mesh, V, F, Q, max_fail_frac=0.0):
    E = oracle.boundary(F, len(V))
    g_ref, a, c, fl = oracle.gradient(V, E, Q)
    g = gwn_mesh.gradient(torch.from_numpy(Q).cuda()).cpu().numpy().astype(np.float64)
    ok = fl == 0
    tol = U * (128.0 * c + 128.0 * a) + 1e-9
    err = np.abs(g - g_ref)
    bad = ok[:, None] & (err > tol[:, None])
    assert not bad.any(), (np.flatnonzero(bad.any(1))[:5], err[bad][:5], tol[bad.any(1)][:5])
    # the bound is informative: over a batch, typical tolerances stay below 5% of
    # typical gradients.  (On a soup with many small holes the terms of each hole's
    # loop cancel into a weak dipole: sum |T| / |grad w| reaches ~2,000 there, and
    # any bound proportional to sum |T| is then a few percent of the result; on the
    # cap it is 4e-4.)  A single query may sit where the terms cancel even more.
    if ok.sum() >= 100:
        mag = np.linalg.norm(g_ref[ok], axis=1)
        assert np.median(tol[ok]) < 5e-2 * np.median(mag) + 1e-9
    print(f"gradient parity: {int(ok.sum())} queries, max err/tol {np.max((err / tol[:, None])[ok]):.3g}, "
          f"median tol/|grad| {np.median(tol[ok] / np.maximum(np.linalg.norm(g_ref[ok], axis=1), 1e-30)):.3g}")
    return g, g_ref, ok


def test_small_cap(gwn):
    mesh, Q = gen.workload("small")
    with gwn.Mesh(mesh.V, mesh.F) as m:
        _check(m, mesh.V, mesh.F, Q)


@pytest.mark.parametrize("n", [1, 300, 20_001])
def test_soup_level5(gwn, n):
    """n = 1 and 300 take the chunk-split path (boundary split across blocks)."""
    mesh, rng = gen.displaced_soup(5, seed=11)
    Q = np.concatenate([gen.queries_uniform_bbox(mesh.V, n - n // 2, rng),
                        gen.queries_near_surface(mesh.V, mesh.F, n // 2, rng)])
    with gwn.Mesh(mesh.V, mesh.F) as m:
        _check(m, mesh.V, mesh.F, Q)


def test_closed_mesh_and_empty(gwn):
    V, F = gen.icosphere(2)
    with gwn.Mesh(V.astype(np.float32), F.astype(np.int32)) as m:
        g = m.gradient(torch.rand((100, 3), device="cuda"))
        assert torch.all(g == 0)
        g0 = m.gradient(torch.zeros((0, 3), device="cuda"))
        assert g0.shape == (0, 3)


def test_query_on_boundary_vertex_is_counted(gwn):
    mesh = gen.small_cap(3, 0.8)
    E = oracle.boundary(mesh.F, mesh.nv)
    Q = mesh.V[E[:5, 0]].copy()
    with gwn.Mesh(mesh.V, mesh.F) as m:
        m.counters(reset=True)
        g = m.gradient(torch.from_numpy(Q).cuda()).cpu().numpy()
        c = m.counters()
        assert c["gradient_skipped"] >= 2 * len(Q)      # both edges at the vertex
        assert np.all(np.isfinite(g))


def test_host_buffers_match_device(gwn):
    mesh, Q = gen.workload("small", n_query=3000)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        gd = m.gradient(torch.from_numpy(Q).cuda()).cpu().numpy()
        gh = m.gradient(Q)
        assert isinstance(gh, np.ndarray) and np.array_equal(gd, gh)


@pytest.mark.slow
def test_soup8_full_size_sampled(gwn):
    """The benchmark's launch: 2M queries on the 2.57M-triangle soup, sampled."""
    mesh, Q = gen.workload("soup8")
    idx = np.random.default_rng(5).choice(len(Q), 1500, replace=False)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        g = m.gradient(torch.from_numpy(Q).cuda()).cpu().numpy().astype(np.float64)[idx]
    E = oracle.boundary(mesh.F, mesh.nv)
    g_ref, a, c, fl = oracle.gradient(mesh.V, E, Q[idx])
    ok = fl == 0
    tol = U * (128.0 * c + 128.0 * a) + 1e-9
    assert not (ok[:, None] & (np.abs(g - g_ref) > tol[:, None])).any()
