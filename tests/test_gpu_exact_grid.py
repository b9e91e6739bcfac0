"""The exact stages of the crossing predicates (Supp. S2.1) on inputs built to
reach them: triangle soups with vertices on a tiny integer grid (collinear,
coplanar, repeated and zero-area triangles included) queried on every point
and half-point of the grid, so that nearly every 2-D edge sign and plane side
is exactly zero before the symbolic perturbation.  On such inputs every
coordinate difference is exact in FP32 and the FP32 error-free stages decide
(also scaled by 2^20); scaled copies whose products leave that stage's safe
range (by 2^-70: below it, by 2^62: above it) and a shift by 1/3 that makes
differences inexact must reach the FP64 expansions.  Compared
bit for bit with the oracle's big-integer predicates."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


def _grid_case(seed, n_tri=300, size=4):
    rng = np.random.default_rng(seed)
    g = np.arange(size + 1, dtype=np.float32)
    P = np.stack(np.meshgrid(g, g, np.array([0.0, 1.0, 2.0], np.float32), indexing="ij"), -1).reshape(-1, 3)
    F = rng.integers(0, len(P), size=(n_tri, 3)).astype(np.int32)
    h = np.arange(0, 2 * size + 1, dtype=np.float32) * 0.5
    Q = np.stack(np.meshgrid(h, h, np.array([-0.5, 0.0, 0.5, 1.0, 1.5], np.float32), indexing="ij"), -1).reshape(-1, 3)
    return P, F, Q


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("scale,shift", [(1.0, 0.0), (2.0 ** 20, 0.0), (2.0 ** -70, 0.0), (2.0 ** 62, 0.0),
                                         (1.0, 1.0 / 3.0)])
def test_exact_stages_on_integer_grids(gwn, seed, scale, shift):
    P, F, Q = _grid_case(seed)
    V = (P.astype(np.float64) * scale + shift).astype(np.float32)
    Qs = (Q.astype(np.float64) * scale + shift).astype(np.float32)
    ref = oracle.chi(V, F, Qs)
    with gwn.Mesh(V, F) as m:
        m.counters(reset=True)
        chi = m.chi(torch.from_numpy(Qs).cuda()).cpu().numpy()
        c = m.counters()
    assert np.array_equal(chi, ref)
    assert c["exact_edge"] > 100 and c["exact_plane"] > 0 and c["error_flags"] == 0
