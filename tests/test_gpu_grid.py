"""Grid queries with ray reuse (Supp. S3) against the per-point path and the oracle.

The grid path decides every cell with the same exact, perturbed predicate the
per-point traversal evaluates at that point, so chi must be bit-identical to
gwn_query_chi on the materialised points and to the oracle's exact chi; the
labels and w of gwn_classify_grid must equal gwn_classify on the same points.
"""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


def _points(x, y, z):
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)


def test_small_cap_matches_points_and_oracle(gwn):
    mesh = gen.small_cap(3, 0.8)
    x = np.linspace(-1.5, 1.5, 40, dtype=np.float32)
    y = np.linspace(-1.4, 1.45, 37, dtype=np.float32)
    z = np.linspace(-1.5, 1.5, 33, dtype=np.float32)
    P = _points(x, y, z)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        g = m.grid_chi(x, y, z).cpu().numpy().ravel()
        per_point = m.chi(torch.from_numpy(P).cuda()).cpu().numpy()
        assert np.array_equal(g, per_point)
        assert np.array_equal(g, oracle.chi(mesh.V, mesh.F, P))
        # host output buffers
        assert np.array_equal(m.grid_chi(x, y, z, device=False).ravel(), g)


def test_integer_grid_on_degenerate_workload(gwn):
    """Cells exactly on vertices, edges and faces of the voxel staircase and the
    integer height field: every tie goes through the perturbation."""
    mesh, _, _ = gen.precision_workload(n_query=1000)
    x = np.arange(-46, 47, 2, dtype=np.float32)
    y = np.arange(-45, 48, 3, dtype=np.float32)
    z = np.arange(-44, 50, 1, dtype=np.float32)
    P = _points(x, y, z)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        m.counters(reset=True)
        g = m.grid_chi(x, y, z).cpu().numpy().ravel()
        c = m.counters()
        per_point = m.chi(torch.from_numpy(P).cuda()).cpu().numpy()
    assert np.array_equal(g, per_point)
    assert c["exact_edge"] + c["exact_plane"] > 0          # the exact fallbacks were exercised
    idx = np.random.default_rng(3).choice(len(P), 3000, replace=False)
    assert np.array_equal(g[idx], oracle.chi(mesh.V, mesh.F, P[idx]))


def test_classify_grid_matches_classify(gwn):
    mesh, _ = gen.displaced_soup(5, seed=12)
    lo, hi = mesh.V.min(0) - 0.1, mesh.V.max(0) + 0.1
    x = np.linspace(lo[0], hi[0], 45, dtype=np.float32)
    y = np.linspace(lo[1], hi[1], 41, dtype=np.float32)
    z = np.linspace(lo[2], hi[2], 39, dtype=np.float32)
    P = torch.from_numpy(_points(x, y, z)).cuda()
    with gwn.Mesh(mesh.V, mesh.F) as m:
        lab_g, w_g = m.classify_grid(x, y, z, want_w=True)
        lab_p, w_p = m.classify(P, want_w=True)
        assert torch.equal(lab_g.ravel(), lab_p)
        assert torch.equal(w_g.ravel(), w_p)
        lab_only = m.classify_grid(x, y, z)
        assert torch.equal(lab_only, lab_g)


def test_closed_mesh(gwn):
    V, F = gen.icosphere(3)
    x = y = z = np.linspace(-1.2, 1.2, 30, dtype=np.float32)
    with gwn.Mesh(V.astype(np.float32), F.astype(np.int32)) as m:
        lab, w = m.classify_grid(x, y, z, want_w=True)
        chi = m.chi(torch.from_numpy(_points(x, y, z)).cuda())
        assert torch.equal(w.ravel(), chi.float())
        assert torch.equal(lab.ravel(), (chi > 0).to(torch.uint8))


def test_deep_column_falls_back_per_cell(gwn):
    """60 stacked squares over one column: more hits than a column keeps, so the
    per-cell walk decides that column; the result is still exact."""
    layers = 60
    V, F = [], []
    for k in range(layers):
        b = len(V)
        zc = float(k)
        V += [[-1, -1, zc], [1, -1, zc], [1, 1, zc], [-1, 1, zc]]
        F += [[b, b + 1, b + 2], [b, b + 2, b + 3]]
    V = np.array(V, np.float32)
    F = np.array(F, np.int32)
    x = np.array([-0.3, 0.25, 2.0], np.float32)
    y = np.array([0.1, -0.7], np.float32)
    z = np.linspace(-1.5, 61.5, 80, dtype=np.float32)
    P = _points(x, y, z)
    with gwn.Mesh(V, F) as m:
        g = m.grid_chi(x, y, z).cpu().numpy().ravel()
        assert np.array_equal(g, m.chi(torch.from_numpy(P).cuda()).cpu().numpy())
    assert np.array_equal(g, oracle.chi(V, F, P))
    assert g.max() == layers


def test_invalid_axes(gwn):
    mesh = gen.small_cap(3, 0.8)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        with pytest.raises(gwn.GwnError) as e:
            m.grid_chi([0.0], [0.0], [1.0, 0.5])
        assert e.value.code == 1
        with pytest.raises(gwn.GwnError):
            m.grid_chi([np.nan], [0.0], [0.0])
        assert m.grid_chi([], [0.0], [0.0]).numel() == 0
