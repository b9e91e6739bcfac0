"""Fixed-point predicates on the GPU (gwn_config.quantize_bits = 30, Supp. S2.1)
against the oracle's fixed-point variant: crossing counts and labels
bit-exact, w within 1e-5."""
import ctypes

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = 1e-5
FIXED = {"quantize_bits": 30}


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


def _compare(m, mesh, Q):
    ref = oracle.reference(mesh.V, mesh.F, Q, quantize_bits=30)
    q = torch.from_numpy(Q).cuda()
    w, chi = m.query(q)
    lab = m.classify(q)
    chi = chi.cpu().numpy()
    assert np.array_equal(chi, ref["chi"])
    ok = ref["flags"] == 0
    dw = np.abs(w.cpu().numpy().astype(np.float64) - ref["w_antipodal"])[ok]
    assert dw.max(initial=0.0) <= TOL_W, dw.max()
    tie = np.abs(ref["w_antipodal"] - 0.5) < 1e-9
    sel = ok & ~tie
    assert np.array_equal(lab.cpu().numpy()[sel], (ref["w_antipodal"][sel] > 0.5).astype(np.uint8))
    return ref


def test_degenerate_workload_matches_oracle_and_exact(gwn):
    mesh, Q, _ = gen.precision_workload(n_query=20_000, seed=7, radius=16.0)
    with gwn.Mesh(mesh.V, mesh.F, config=FIXED) as m:
        ref = _compare(m, mesh, Q)
    # integer inputs: snapping is exact, so the exact predicates agree everywhere
    assert np.array_equal(ref["chi"], oracle.chi(mesh.V, mesh.F, Q))


def test_random_soup(gwn):
    mesh, rng = gen.displaced_soup(5, seed=41)
    Q = np.concatenate([gen.queries_uniform_bbox(mesh.V, 10_000, rng),
                        gen.queries_near_surface(mesh.V, mesh.F, 10_000, rng)])
    with gwn.Mesh(mesh.V, mesh.F, config=FIXED) as m:
        _compare(m, mesh, Q)


def test_snapping_changes_the_crossing_within_one_quantum(gwn):
    """Half-extent 4 gives the quantum 2^-26: a square 2^-30 above the query
    snaps onto its height (no crossing); the exact predicates see it above."""
    h = 2.0 ** -30
    V = np.array([[-1, -1, h], [1, -1, h], [1, 1, h], [-1, 1, h], [-3, 0, -4], [5, 0, 4]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    q = torch.tensor([[0.25, 0.1, 0.0]], dtype=torch.float32, device="cuda")
    with gwn.Mesh(V, F, config=FIXED) as m:
        assert int(m.chi(q).item()) == 0
    with gwn.Mesh(V, F) as m:
        assert int(m.chi(q).item()) == 1


def test_batch_and_static_paths(gwn):
    mesh, rng = gen.displaced_soup(4, seed=43)
    Q = np.concatenate([gen.queries_uniform_bbox(mesh.V, 3000, rng),
                        gen.queries_near_surface(mesh.V, mesh.F, 3000, rng)])
    q = torch.from_numpy(Q).cuda()
    with gwn.Mesh(mesh.V, mesh.F, config=FIXED) as m:
        w_ref, chi_ref = m.query(q)
        lab_ref = m.classify(q)
        with gwn.Batch([m], [len(Q)]) as b:
            w, chi = b.run(q)
            torch.cuda.synchronize()
            assert torch.equal(chi, chi_ref)
            assert torch.max(torch.abs(w - w_ref)).item() <= TOL_W
        lib = gwn.load()
        lab = torch.empty(len(Q), dtype=torch.uint8, device="cuda")
        rc = lib.gwn_classify_static(m.handle, ctypes.c_void_p(q.data_ptr()), len(Q), ctypes.c_void_p(lab.data_ptr()),
                                     None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, lib.gwn_last_error()
        torch.cuda.synchronize()
        assert torch.equal(lab, lab_ref)


def test_grid_entry_points_refuse_fixed_meshes(gwn):
    mesh = gen.small_cap(3, 0.8)
    with gwn.Mesh(mesh.V, mesh.F, config=FIXED) as m:
        with pytest.raises(gwn.GwnError) as e:
            m.grid_chi([0.0], [0.0], [0.0])
        assert e.value.code == 1


def test_invalid_bits(gwn):
    mesh = gen.small_cap(3, 0.8)
    with pytest.raises(gwn.GwnError) as e:
        gwn.Mesh(mesh.V, mesh.F, config={"quantize_bits": 20})
    assert e.value.code == 1
