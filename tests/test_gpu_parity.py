"""GPU parity tests: the CUDA library through its C ABI against the CPU oracle.

Bars (fixed here, not loosened per case):
* boundary edges, crossing numbers chi and labels: bit-exact;
* w (antipodal and direct, FP32): |w_gpu - w_oracle| <= 1e-5 absolute.
Queries the oracle flags as lying on the boundary curve (w undefined there) are
excluded from the w and label comparisons and counted; their chi is still
compared.  Labels whose oracle w lies within 1e-9 of 1/2 are ties (excluded).
"""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = 1e-5


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _compare(m, mesh, Q, ref, check_direct=True, tol=TOL_W):
    q = _cuda(Q)
    w, chi = m.query(q)
    lab, wc = m.classify(q, want_w=True)
    torch.cuda.synchronize()
    chi = chi.cpu().numpy()
    w = w.cpu().numpy().astype(np.float64)
    wc = wc.cpu().numpy().astype(np.float64)
    lab = lab.cpu().numpy()
    assert np.array_equal(chi, ref["chi"]), f"chi mismatches: {int((chi != ref['chi']).sum())}"
    ok = ref["flags"] == 0
    dw = np.abs(w - ref["w_antipodal"])[ok]
    assert dw.size == 0 or dw.max() <= tol, f"max |dw| = {dw.max():.3e}"
    dwc = np.abs(wc - ref["w_antipodal"])[ok]
    assert dwc.size == 0 or dwc.max() <= tol
    tie = np.abs(ref["w_antipodal"] - 0.5) < 1e-9
    sel = ok & ~tie
    assert np.array_equal(lab[sel], (ref["w_antipodal"][sel] > 0.5).astype(np.uint8))
    if check_direct and "w_direct" in ref:
        wd = m.direct(q).cpu().numpy().astype(np.float64)
        fin = ok & np.isfinite(ref["w_direct"])
        dd = np.abs(wd - ref["w_direct"])[fin]
        assert dd.max() <= tol, f"direct max |dw| = {dd.max():.3e}"
    return {"max_dw": float(dw.max()) if dw.size else 0.0, "excluded": int((~ok).sum())}


def test_small_cap_full(gwn):
    mesh, Q = gen.workload("small")
    ref = oracle.reference(mesh.V, mesh.F, Q, with_direct=True)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        assert np.array_equal(m.boundary_edges(), ref["edges"])
        info = m.info()
        assert info["n_boundary_edges"] == 36 and info["n_boundary_loops"] == 1
        _compare(m, mesh, Q, ref)


@pytest.mark.parametrize("cfg", [dict(), dict(queries_per_thread=1), dict(queries_per_thread=2),
                                 dict(queries_per_thread=8), dict(chain_boundary=-1),
                                 dict(boundary_tile=96, queries_per_thread=2)])
def test_soup_level5_configs(gwn, cfg):
    """Displaced self-intersecting soup with holes (level 5: 2 x 20480 faces, 2%
    holes): several tiles of boundary points, a ragged query count."""
    mesh, rng = gen.displaced_soup(5, seed=11)
    Q = np.concatenate([gen.queries_uniform_bbox(mesh.V, 1777, rng),
                        gen.queries_near_surface(mesh.V, mesh.F, 1777, rng)])
    ref = oracle.reference(mesh.V, mesh.F, Q, with_direct=True)
    with gwn.Mesh(mesh.V, mesh.F, config=cfg) as m:
        assert np.array_equal(m.boundary_edges(), ref["edges"])
        info = m.info()
        assert info["n_boundary_points"] == (2 * info["n_boundary_edges"] if cfg.get("chain_boundary") == -1
                                             else info["n_boundary_edges"] + info["n_boundary_loops"])
        _compare(m, mesh, Q, ref)


def _edge_position_multiset(V, E):
    P = V[E.reshape(-1)].reshape(-1, 6)
    return sorted(map(tuple, P.tolist()))


@pytest.mark.parametrize("level", [3, 6, 8])
def test_chained_points_reproduce_boundary(gwn, level):
    """The chained point stream holds exactly the oriented boundary edges: every
    flagged consecutive pair is an edge of dM and the multiset is dM."""
    mesh, _ = gen.displaced_soup(level, seed=4)
    E = oracle.boundary(mesh.F, mesh.nv)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        P = m.boundary_points()
        info = m.info()
    assert len(P) == info["n_boundary_edges"] + info["n_boundary_loops"]
    j = np.where(P[:-1, 3] != 0)[0]
    got = np.concatenate([P[j, :3], P[j + 1, :3]], axis=1)
    assert len(j) == len(E)
    assert sorted(map(tuple, got.tolist())) == _edge_position_multiset(mesh.V, E)
    # every loop is closed: the point after a loop's last edge repeats its first point
    starts = np.concatenate([[0], np.where(P[:, 3] == 0)[0][:-1] + 1])
    ends = np.where(P[:, 3] == 0)[0]
    assert np.array_equal(P[starts, :3], P[ends, :3])


def test_tiny_terms_straight_above_query(gwn):
    """Many small holes almost straight above the query: each boundary term has
    |d + i n| ~ 1e-4, so a group of eight multiplies down to ~1e-31 (a normal
    float).  The group's angle must still be exact (this failed once when the
    atan2 denominator was clamped at 1e-30)."""
    rng = np.random.default_rng(17)
    k = 400
    c = np.stack([rng.uniform(-0.03, 0.03, k), rng.uniform(-0.03, 0.03, k), np.full(k, 2.0)], 1)
    e1 = rng.normal(size=(k, 3)) * 0.004
    e2 = rng.normal(size=(k, 3)) * 0.004
    V = np.stack([c, c + e1, c + e2], 1).reshape(-1, 3).astype(np.float32)
    F = np.arange(3 * k, dtype=np.int32).reshape(-1, 3)
    Q = np.stack([rng.uniform(-0.02, 0.02, 300), rng.uniform(-0.02, 0.02, 300), rng.uniform(-0.2, 0.2, 300)],
                 1).astype(np.float32)
    ref = oracle.reference(V, F, Q, with_direct=True)
    with gwn.Mesh(V, F) as m:
        _compare(m, None, Q, ref)


def test_few_queries_split_boundary(gwn):
    """Few queries against a long boundary: the boundary sum is split into point
    chunks with FP64 partials combined in order (and the direct sum into triangle
    chunks); results must not depend on the split."""
    mesh, rng = gen.displaced_soup(6, seed=13)
    Q = np.concatenate([gen.queries_uniform_bbox(mesh.V, 751, rng),
                        gen.queries_near_surface(mesh.V, mesh.F, 750, rng)])
    ref = oracle.reference(mesh.V, mesh.F, Q, with_direct=True)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        assert m.info()["n_boundary_points"] > 8 * 1024      # several chunks of 2 tiles
        _compare(m, mesh, Q, ref)
        # one query at a time gives the same w as the batch (up to FP64 summation order)
        w_all, _ = m.query(_cuda(Q[:64]))
        for i in range(0, 64, 16):
            w1, _ = m.query(_cuda(Q[i:i + 1]))
            assert abs(float(w1.item()) - float(w_all[i].item())) <= 1e-6


def test_precision_workload_reduced(gwn):
    """Integer staircase + height field with exact degenerate queries (vertices,
    edge midpoints, face points, grid points): chi bit-exact on every query."""
    mesh, Q, kinds = gen.precision_workload(n_query=4000, seed=5, radius=12.0)
    ref = oracle.reference(mesh.V, mesh.F, Q)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        assert np.array_equal(m.boundary_edges(), ref["edges"])
        r = _compare(m, mesh, Q, ref, check_direct=False)
        c = m.counters()
    assert c["error_flags"] == 0
    assert c["exact_edge"] > 0 and c["exact_plane"] > 0   # the exact paths were exercised


def test_random_meshes_bit_exact_boundary(gwn):
    rng = np.random.default_rng(8)
    for trial in range(20):
        nv = int(rng.integers(3, 60))
        nt = int(rng.integers(1, 200))
        F = rng.integers(0, nv, size=(nt, 3)).astype(np.int32)   # repeated indices allowed
        V = rng.normal(size=(nv, 3)).astype(np.float32)
        Q = rng.normal(size=(300, 3)).astype(np.float32)
        ref = oracle.reference(V, F, Q)
        with gwn.Mesh(V, F) as m:
            assert np.array_equal(m.boundary_edges(), ref["edges"])
            q = _cuda(Q)
            w, chi = m.query(q)
            assert np.array_equal(chi.cpu().numpy(), ref["chi"])
            ok = ref["flags"] == 0
            assert np.abs(w.cpu().numpy() - ref["w_antipodal"])[ok].max() <= TOL_W


def test_edge_cases(gwn):
    # closed mesh: no boundary, w == chi
    V, F = gen.icosphere(2)
    V = V.astype(np.float32); F = F.astype(np.int32)
    Q = np.random.default_rng(1).uniform(-1.5, 1.5, (1000, 3)).astype(np.float32)
    ref = oracle.reference(V, F, Q)
    with gwn.Mesh(V, F) as m:
        assert m.info()["n_boundary_edges"] == 0
        w, chi = m.query(_cuda(Q))
        assert np.array_equal(chi.cpu().numpy(), ref["chi"])
        assert np.array_equal(w.cpu().numpy(), ref["chi"].astype(np.float32))
        # empty query batch
        w0, c0 = m.query(torch.zeros((0, 3), dtype=torch.float32, device="cuda"))
        assert w0.numel() == 0 and c0.numel() == 0
        # single query
        w1, c1 = m.query(_cuda(Q[:1]))
        assert int(c1.item()) == int(ref["chi"][0])
    # single triangle
    V1 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F1 = np.array([[0, 1, 2]], np.int32)
    ref = oracle.reference(V1, F1, Q, with_direct=True)
    with gwn.Mesh(V1, F1) as m:
        _compare(m, None, Q, ref)
    # empty mesh
    with gwn.Mesh(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32)) as m:
        w, chi = m.query(_cuda(Q[:10]))
        assert torch.all(w == 0) and torch.all(chi == 0)
    # degenerate faces (repeated indices, collinear points) are allowed
    V2 = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0]], np.float32)
    F2 = np.array([[0, 1, 2], [0, 0, 3], [0, 1, 3]], np.int32)
    ref = oracle.reference(V2, F2, Q)
    with gwn.Mesh(V2, F2) as m:
        assert np.array_equal(m.boundary_edges(), ref["edges"])
        w, chi = m.query(_cuda(Q))
        assert np.array_equal(chi.cpu().numpy(), ref["chi"])


def test_invalid_inputs_fail_loudly(gwn):
    V = np.zeros((3, 3), np.float32)
    with pytest.raises(gwn.GwnError) as e:
        gwn.Mesh(V, np.array([[0, 1, 3]], np.int32))
    assert e.value.code == 2
    Vn = V.copy(); Vn[1, 1] = np.nan
    with pytest.raises(gwn.GwnError):
        gwn.Mesh(Vn, np.array([[0, 1, 2]], np.int32))
    with gwn.Mesh(V, np.array([[0, 1, 2]], np.int32), build=False) as m:
        with pytest.raises(gwn.GwnError) as e:
            m.query(torch.zeros((4, 3), device="cuda"))
        assert e.value.code == 3


def test_host_buffers_match_device(gwn):
    mesh, Q = gen.workload("small", n_query=5000)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        wd, cd = m.query(_cuda(Q))
        wh, ch = m.query(Q)                       # numpy: staged by the library
        qp = torch.from_numpy(Q).pin_memory()
        wp, cp = m.query(qp)                      # pinned host tensor
        assert isinstance(wh, np.ndarray) and wp.is_pinned()
        assert np.array_equal(wd.cpu().numpy(), wh) and np.array_equal(cd.cpu().numpy(), ch)
        assert np.array_equal(wh, wp.numpy()) and np.array_equal(ch, cp.numpy())
        lh = m.classify(Q)
        ld = m.classify(_cuda(Q)).cpu().numpy()
        assert np.array_equal(lh, ld)


@pytest.mark.slow
def test_soup8_full_size_sampled(gwn):
    """The benchmark workload (2.57M triangles, 154k boundary edges, 2M queries)
    in the benchmark's launch configuration; a seeded sample against the oracle."""
    mesh, Q = gen.workload("soup8")
    with gwn.Mesh(mesh.V, mesh.F) as m:
        lab, w = m.classify(_cuda(Q), want_w=True)
        _, chi = m.query(_cuda(Q))
        torch.cuda.synchronize()
        lab, w, chi = lab.cpu().numpy(), w.cpu().numpy(), chi.cpu().numpy()
    idx = np.random.default_rng(0).choice(len(Q), 800, replace=False)
    ref = oracle.reference(mesh.V, mesh.F, Q[idx])
    assert np.array_equal(chi[idx], ref["chi"])
    ok = ref["flags"] == 0
    assert np.abs(w[idx] - ref["w_antipodal"])[ok].max() <= TOL_W
    tie = np.abs(ref["w_antipodal"] - 0.5) < 1e-9
    assert np.array_equal(lab[idx][ok & ~tie], (ref["w_antipodal"] > 0.5)[ok & ~tie])


@pytest.mark.slow
def test_soup7_full_size_sampled(gwn):
    """The 642k-triangle soup with 2M queries in the launch configuration the
    benchmark uses; the oracle checks a seeded sample of outputs."""
    mesh, Q = gen.workload("soup7")
    with gwn.Mesh(mesh.V, mesh.F) as m:
        assert np.array_equal(m.boundary_edges(), oracle.boundary(mesh.F, mesh.nv))
        lab, w = m.classify(_cuda(Q), want_w=True)
        _, chi = m.query(_cuda(Q))
        torch.cuda.synchronize()
        lab, w, chi = lab.cpu().numpy(), w.cpu().numpy(), chi.cpu().numpy()
    idx = np.random.default_rng(0).choice(len(Q), 600, replace=False)
    ref = oracle.reference(mesh.V, mesh.F, Q[idx])
    assert np.array_equal(chi[idx], ref["chi"])
    ok = ref["flags"] == 0
    assert np.abs(w[idx] - ref["w_antipodal"])[ok].max() <= TOL_W
    tie = np.abs(ref["w_antipodal"] - 0.5) < 1e-9
    assert np.array_equal(lab[idx][ok & ~tie], (ref["w_antipodal"] > 0.5)[ok & ~tie])


@pytest.mark.gpu
def test_instrumented_walk_counts_and_matches():
    """gwn_query_chi_visits: the same crossing counts as gwn_query_chi, and visit
    totals that bound what the walk must read (at least one node per query, and
    at least the crossings' triangles)."""
    import gen
    import paper_2605_01536_gb300 as gwn
    mesh, Q = gen.workload("small", n_query=4096)
    q = torch.from_numpy(Q).cuda()
    with gwn.Mesh(mesh.V, mesh.F) as m:
        chi = m.chi(q)
        chi2, nodes, tris = m.chi_visits(q)
        assert torch.equal(chi, chi2)
        assert nodes >= len(Q)
        assert tris >= int(torch.abs(chi).sum().item())
        # the counts are totals of one walk per query: independent of batching
        _, n1, t1 = m.chi_visits(q[:1000])
        _, n2, t2 = m.chi_visits(q[1000:])
        assert (n1 + n2, t1 + t2) == (nodes, tris)
        # host queries are staged through the device: same counts
        chi_h, nh, th = m.chi_visits(Q)
        assert np.array_equal(chi_h, chi.cpu().numpy()) and (nh, th) == (nodes, tris)


def test_results_do_not_depend_on_query_order(gwn):
    """Each query's boundary terms take the same decisions whichever warp it
    shares (the cancellation-checking loop runs only for warps near a tile, and
    no query far from it has a term that loop would treat differently), so w
    is bit-identical in Morton order and in the caller's order (gwn_classify
    against gwn_classify_static) and in a shuffled order (gwn_query_batch).  Dense random
    soup, half the queries within 1e-6..3e-5 edge lengths of its edges."""
    import ctypes
    rng = np.random.default_rng(21)
    mesh = gen.random_soup(20_000, rng)
    near = gen.queries_near_triangle_edges(mesh.V, mesh.F, 20_000, rng)
    Q = np.concatenate([near, gen.queries_uniform_bbox(mesh.V, 20_000, rng)]).astype(np.float32)
    perm = rng.permutation(len(Q))
    with gwn.Mesh(mesh.V, mesh.F) as m:
        q = _cuda(Q)
        lab, w = m.classify(q, want_w=True)
        wq, chi = m.query(q)
        wp, chip = m.query(_cuda(Q[perm]))
        lab_s = torch.empty(len(Q), dtype=torch.uint8, device="cuda")
        w_s = torch.empty(len(Q), dtype=torch.float32, device="cuda")
        lib = gwn.load()
        rc = lib.gwn_classify_static(m.handle, ctypes.c_void_p(q.data_ptr()), len(Q), ctypes.c_void_p(lab_s.data_ptr()),
                                     ctypes.c_void_p(w_s.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, lib.gwn_last_error()
        torch.cuda.synchronize()
        c = m.counters()
    w, wq, w_s = w.cpu().numpy(), wq.cpu().numpy(), w_s.cpu().numpy()
    back = np.empty_like(w)
    back[perm] = wp.cpu().numpy()
    assert c["cancel_terms"] > 0                      # the FP64 terms were exercised
    assert np.array_equal(w, w_s)                     # classify: Morton order vs the caller's
    assert np.array_equal(wq, back)                   # query_batch: two orders
    # classify re-evaluates queries within 1e-4 of 1/2 in FP64; the rest is the same sum
    keep = np.abs(wq.astype(np.float64) - 0.5) > 2e-4
    assert np.array_equal(w[keep], wq[keep])
    assert torch.equal(lab, lab_s)
    chi_back = np.empty_like(chi.cpu().numpy())
    chi_back[perm] = chip.cpu().numpy()
    assert np.array_equal(chi.cpu().numpy(), chi_back)


@pytest.mark.parametrize("which", ["soup", "cap"])
def test_group_tests_agree(gwn, which):
    """Both group acceptance tests of the boundary kernel (gwn_config.group_test
    1: each angle below pi/8; 2: the running product keeps a positive real
    part) against the oracle, on a random soup (dense boundary: the default
    picks the running test; many steep terms exercise it) and on the small cap
    (the default picks the per-term test): crossing numbers and labels
    bit-exact, w within 1e-5 for both and for the default.  Values outside
    0..2 are rejected."""
    rng = np.random.default_rng(31)
    if which == "soup":
        mesh = gen.random_soup(4000, rng)
        Q = np.concatenate([gen.queries_near_surface(mesh.V, mesh.F, 3000, rng),
                            gen.queries_uniform_bbox(mesh.V, 3000, rng)]).astype(np.float32)
    else:
        mesh = gen.small_cap()
        Q = gen.queries_uniform_bbox(mesh.V, 6000, rng).astype(np.float32)
    ref = oracle.reference(mesh.V, mesh.F, Q)
    ws = {}
    for flag in (0, 1, 2):
        with gwn.Mesh(mesh.V, mesh.F, config={"group_test": flag}) as m:
            _compare(m, mesh, Q, ref, check_direct=False)
            w, _ = m.query(_cuda(Q))
            ws[flag] = w.cpu().numpy()
    auto = 2 if which == "soup" else 1
    assert np.array_equal(ws[0], ws[auto])
    for bad in (-1, 3):
        with pytest.raises(gwn.GwnError):
            gwn.Mesh(mesh.V, mesh.F, config={"group_test": bad})
