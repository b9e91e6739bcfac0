"""FP64 re-evaluation of boundary terms whose denominator cancels
(gwn_config.fp64_cancel = 1) against the FP64 oracle, on queries between 1e-6
and 3e-5 edge lengths from boundary edges of a random soup: there the FP32
term's rounding grows like the edge length over the distance (the plain path
misses |dw| <= 1e-5 on most of them), and the re-evaluated sum must stay
within 2e-6.  Crossing counts bit-exact on both paths, labels on the
re-evaluated one (also through the allocation-free classify)."""
import ctypes

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


@pytest.mark.parametrize("seed", [11, 12])
def test_cancelling_terms_in_fp64(gwn, seed):
    rng = np.random.default_rng(seed)
    mesh = gen.random_soup(400, rng)
    Q = gen.queries_near_triangle_edges(mesh.V, mesh.F, 64, rng)
    ref = oracle.reference(mesh.V, mesh.F, Q)
    ok = ref["flags"] == 0
    assert ok.sum() >= 48
    q = torch.from_numpy(Q).cuda()
    err = {}
    for flag in (0, 1):
        with gwn.Mesh(mesh.V, mesh.F, config={"fp64_cancel": flag}) as m:
            w, chi = m.query(q)
            lab = m.classify(q)
            torch.cuda.synchronize()
            assert np.array_equal(chi.cpu().numpy(), ref["chi"])
            err[flag] = np.abs(w.cpu().numpy().astype(np.float64) - ref["w_antipodal"])[ok]
            if flag:
                want = (ref["w_antipodal"] > 0.5).astype(np.uint8)
                assert np.array_equal(lab.cpu().numpy()[ok], want[ok])
                lib = gwn.load()
                lab_s = torch.empty(len(Q), dtype=torch.uint8, device="cuda")
                rc = lib.gwn_classify_static(m.handle, ctypes.c_void_p(q.data_ptr()), len(Q),
                                             ctypes.c_void_p(lab_s.data_ptr()), None,
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
                assert rc == 0, lib.gwn_last_error()
                torch.cuda.synchronize()
                assert torch.equal(lab_s, lab)
    assert (err[0] > 1e-5).sum() >= 10, err[0]        # the case is ill-conditioned for plain FP32
    assert err[1].max() <= 2e-6, err[1].max()


def test_fp64_cancel_must_be_0_or_1(gwn):
    mesh = gen.small_cap(2, 0.8)
    with pytest.raises(gwn.GwnError):
        gwn.Mesh(mesh.V, mesh.F, config={"fp64_cancel": 2})
