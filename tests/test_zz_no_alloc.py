"""gwn_classify_static: the classify path with no device allocation.

Callers that cannot allocate device memory while they run (a fixed, fully
reserved device-memory budget, or a latency-critical loop that must stay out
of the CUDA allocator) use this entry point; its scratch is a file-scope
device array inside the library.  This test calls it through the C ABI and
checks it against gwn_classify on the same inputs, on two calls in a row (the
second call reuses the shared scratch the first one left behind), plus the
size limit.  Collected last on purpose: it runs after every other test, and
also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = 1e-5
MAX_QUERIES = 2_097_152


def _classify(lib, fn, h, q, stream):
    n = q.shape[0]
    label = torch.empty(n, dtype=torch.uint8, device=q.device)
    w = torch.empty(n, dtype=torch.float32, device=q.device)
    rc = getattr(lib, fn)(h, ctypes.c_void_p(q.data_ptr()), n, ctypes.c_void_p(label.data_ptr()),
                          ctypes.c_void_p(w.data_ptr()), stream)
    assert rc == 0, (fn, rc, lib.gwn_last_error())
    torch.cuda.synchronize()
    return label.cpu().numpy(), w.cpu().numpy()


def test_classify_static_matches_classify_twice():
    import paper_2605_01536_gb300 as gwn
    lib = gwn.load()
    mesh, rng = gen.displaced_soup(6, seed=21)
    sets = [
        np.concatenate([gen.queries_uniform_bbox(mesh.V, 1500, rng), gen.queries_near_surface(mesh.V, mesh.F, 1501, rng)]),
        np.concatenate([gen.queries_uniform_bbox(mesh.V, 150000, rng), gen.queries_near_surface(mesh.V, mesh.F, 150000, rng)]),
        # exactly at the static scratch limit: the unsplit path with the whole array in use
        np.concatenate([gen.queries_uniform_bbox(mesh.V, MAX_QUERIES // 2, rng),
                        gen.queries_near_surface(mesh.V, mesh.F, MAX_QUERIES // 2, rng)]),
    ]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with gwn.Mesh(mesh.V, mesh.F) as m:
        for Q in sets:
            q = torch.from_numpy(Q).cuda()
            lab_ref, w_ref = _classify(lib, "gwn_classify", m.handle, q, stream)
            for _ in range(2):   # two calls in a row on the shared static scratch
                lab, w = _classify(lib, "gwn_classify_static", m.handle, q, stream)
                assert np.array_equal(lab, lab_ref)
                assert np.max(np.abs(w.astype(np.float64) - w_ref)) <= TOL_W
        # sizes beyond the static scratch are refused before any work is queued
        q1 = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
        rc = lib.gwn_classify_static(m.handle, ctypes.c_void_p(q1.data_ptr()), MAX_QUERIES + 1,
                                     ctypes.c_void_p(q1.data_ptr()), None, stream)
        assert rc == 1 and b"2097152" in lib.gwn_last_error()
        # host buffers would need staging (an allocation): refused
        qh = np.zeros((4, 3), np.float32)
        lh = np.zeros(4, np.uint8)
        rc = lib.gwn_classify_static(m.handle, qh.ctypes.data_as(ctypes.c_void_p), 4,
                                     lh.ctypes.data_as(ctypes.c_void_p), None, stream)
        assert rc == 1
