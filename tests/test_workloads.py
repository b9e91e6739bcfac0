"""The seeded workloads keep the sizes the design documents and the benchmark
lines quote (no GPU): the generators in gen/ are the only source of inputs for
both the tests and bench.py, so a change to one of them shows up here first."""
import numpy as np
import pytest

import gen
import oracle


@pytest.mark.parametrize("name, n_tri, n_edges", [
    ("small", 1148, 36),
    ("soup7", 642231, 38643),
    ("soup8", 2569061, 153991),
])
def test_named_meshes(name, n_tri, n_edges):
    m, Q = gen.workload(name, n_query=1000)
    assert m.nt == n_tri
    assert len(oracle.boundary(m.F, m.nv)) == n_edges
    assert Q.shape == (1000, 3) and Q.dtype == np.float32


def test_batched_workload_totals():
    items = gen.batched_workload(n_mesh=256, seed=3)
    assert len(items) == 256
    assert sum(m.nt for m, _ in items) == 16_384_894
    assert sum(len(Q) for _, Q in items) == 36_568_668


def test_queries_near_triangle_edges_geometry():
    rng = np.random.default_rng(11)
    m = gen.random_soup(400, rng)
    Q = gen.queries_near_triangle_edges(m.V, m.F, 64, rng).astype(np.float64)
    V = m.V.astype(np.float64)
    # every point lies 10^[-6, -4.5] edge lengths from some triangle edge's interior
    a = V[m.F[:, [0, 1, 2]]].reshape(-1, 3)
    b = V[m.F[:, [1, 2, 0]]].reshape(-1, 3)
    e = b - a
    L = np.linalg.norm(e, axis=1)
    for q in Q:
        t = np.clip(np.sum((q - a) * e, 1) / (L * L), 0, 1)
        d = np.linalg.norm(a + t[:, None] * e - q, axis=1)
        k = np.argmin(d / L)
        assert 0.2 - 1e-6 <= t[k] <= 0.8 + 1e-6
        # the FP32 rounding of the point (below 1e-7 absolute here) widens the band
        assert 1e-6 * L[k] - 1e-7 <= d[k] <= 10 ** -4.5 * L[k] + 1e-7
