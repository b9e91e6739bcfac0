"""CPU oracle for generalized winding numbers (TEST INFRASTRUCTURE ONLY).

The oracle is the plain, slow, obviously-correct reference that the CUDA library
is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import it.  It
shares no code with the library: its arithmetic lives in ``gwn_oracle.c``
(compiled with gcc, OpenMP over queries, FP64 + exact big-integer predicates)
and this module only marshals numpy arrays through ctypes.

Functions and the paper passages they follow (arXiv 2605.01536):

* :func:`direct` - Eqs. 1-2 (Sec. 3.1) with the van Oosterom-Strackee area (Eq. 6) of
  Sec. 3.3, FP64, double-double accumulation (Sec. 5.2 ground-truth protocol).
* :func:`chi` - signed ray crossings (Sec. 3.2) along +z with the exact,
  symbolically perturbed predicates of Supp. S2.1.
* :func:`boundary` - the oriented boundary dM left after interior edges cancel
  (Sec. 4.1).
* :func:`gradient` - Supp. S4, Algorithm 3 (gradient of w), FP64, any antipode.
* ``quantize_bits=30`` in :func:`chi` / :func:`antipodal`: the same predicates on
  inputs snapped to a 30-bit fixed-point grid (Supp. S2.1), 128-bit integers.
* :func:`antipodal` - Eq. 9 / Algorithm 1 with x0 = +z, x1 = -z, FP64, exact
  branch-cut signs (Supp. S2.1).

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force on tiny inputs, or invariants (see each test's
docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwn_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gwn_oracle.c`` into ``oracle/_lib/liboracle.so`` with gcc.

    Contraction of a*b+c into FMA is disabled so that the double-double
    accumulator and every FP64 expression run exactly as written."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_chi.argtypes = [P, I64, P, I64, P, I64, P]
            lib.oracle_direct.argtypes = [P, I64, P, I64, P, I64, P]
            lib.oracle_boundary.argtypes = [P, I64, I64, P]
            lib.oracle_boundary.restype = I64
            lib.oracle_antipodal.argtypes = [P, I64, P, I64, P, I64, P, P, P]
            lib.oracle_chi_fixed.argtypes = [P, I64, P, I64, P, I64, P]
            lib.oracle_antipodal_fixed.argtypes = [P, I64, P, I64, P, I64, P, P, P]
            lib.oracle_gradient.argtypes = [P, I64, P, I64, P, I64, P, P, P, P, P]
            lib.oracle_edge_sos.argtypes = [ctypes.c_float] * 6
            lib.oracle_edge_sos.restype = ctypes.c_int
            lib.oracle_plane_sos.argtypes = [P, P, P, P]
            lib.oracle_plane_sos.restype = ctypes.c_int
            lib.oracle_tri_crossing.argtypes = [P, P, P, P]
            lib.oracle_tri_crossing.restype = ctypes.c_int
            lib.oracle_triangle_area.argtypes = [P, P, P, P]
            lib.oracle_triangle_area.restype = ctypes.c_double
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f32(a, shape_tail=3):
    a = np.ascontiguousarray(a, dtype=np.float32)
    assert a.ndim == 2 and a.shape[1] == shape_tail, a.shape
    return a


def _i32(a, shape_tail):
    a = np.ascontiguousarray(a, dtype=np.int32)
    assert a.ndim == 2 and a.shape[1] == shape_tail, a.shape
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def direct(V, F, Q) -> np.ndarray:
    """w(q) by the direct solid-angle sum, FP64 (float64[n])."""
    V, F, Q = _f32(V), _i32(F, 3), _f32(Q)
    out = np.empty(Q.shape[0], dtype=np.float64)
    _load().oracle_direct(_p(V), V.shape[0], _p(F), F.shape[0], _p(Q), Q.shape[0], _p(out))
    return out


def _check_bits(quantize_bits):
    if quantize_bits not in (0, 30):
        raise ValueError("quantize_bits must be 0 (exact FP32 inputs) or 30 (fixed point)")


def chi(V, F, Q, quantize_bits: int = 0) -> np.ndarray:
    """Exact perturbed signed crossing count along +z (int32[n]); with
    quantize_bits = 30 the predicates are decided on the inputs snapped to the
    mesh's 30-bit fixed-point grid (Supp. S2.1)."""
    _check_bits(quantize_bits)
    V, F, Q = _f32(V), _i32(F, 3), _f32(Q)
    out = np.empty(Q.shape[0], dtype=np.int32)
    fn = _load().oracle_chi_fixed if quantize_bits else _load().oracle_chi
    fn(_p(V), V.shape[0], _p(F), F.shape[0], _p(Q), Q.shape[0], _p(out))
    return out


def boundary(F, nv: int) -> np.ndarray:
    """Oriented boundary edges (int32[B, 2]), sorted by undirected (min, max) key."""
    F = _i32(F, 3)
    out = np.empty((max(3 * F.shape[0], 1), 2), dtype=np.int32)
    nb = _load().oracle_boundary(_p(F), F.shape[0], int(nv), _p(out))
    return out[:nb].copy()


def antipodal(V, E, Q, chi_values, quantize_bits: int = 0):
    """(w float64[n], flags int32[n]) by Eq. 9 with x1 = (0, 0, -1).

    flags bit 0: query on the boundary curve (w undefined);
    flags bit 1: a vertical boundary edge lies on the query's vertical line.
    quantize_bits = 30 takes the branch-cut signs on the snapped integers."""
    _check_bits(quantize_bits)
    V, Q = _f32(V), _f32(Q)
    E = _i32(E.reshape(-1, 2) if len(E) else np.zeros((0, 2), np.int32), 2)
    c = np.ascontiguousarray(chi_values, dtype=np.int32)
    w = np.empty(Q.shape[0], dtype=np.float64)
    fl = np.empty(Q.shape[0], dtype=np.int32)
    fn = _load().oracle_antipodal_fixed if quantize_bits else _load().oracle_antipodal
    fn(_p(V), V.shape[0], _p(E), E.shape[0], _p(Q), Q.shape[0], _p(c), _p(w), _p(fl))
    return w, fl


def gradient(V, E, Q, x1=(0.0, 0.0, -1.0)):
    """(grad float64[n, 3], abs_sum float64[n], cond_sum float64[n], flags int32[n])
    by Supp. S4, Algorithm 3 with antipode x1 (default -z, the library's).

    abs_sum = (1/4pi) sum |term|, cond_sum = (1/4pi) sum |term| / rho with rho the
    unit-vector modulus sqrt(n^2 + d^2) / (l0 l1) of the edge's VOS pair (they
    size the FP32 error bound of a GPU evaluation).  flags bit 0: the query is on
    a boundary segment; bit 1: a term with rho = 0 was skipped."""
    V, Q = _f32(V), _f32(Q)
    E = _i32(E.reshape(-1, 2) if len(E) else np.zeros((0, 2), np.int32), 2)
    x = np.ascontiguousarray(x1, dtype=np.float64).reshape(3)
    g = np.empty((Q.shape[0], 3), dtype=np.float64)
    a = np.empty(Q.shape[0], dtype=np.float64)
    c = np.empty(Q.shape[0], dtype=np.float64)
    fl = np.empty(Q.shape[0], dtype=np.int32)
    _load().oracle_gradient(_p(V), V.shape[0], _p(E), E.shape[0], _p(Q), Q.shape[0], _p(x), _p(g), _p(a), _p(c),
                            _p(fl))
    return g, a, c, fl


def edge_sos(q, pi, pj) -> int:
    """Perturbed sign of the 2-D classification of q against edge pi -> pj."""
    f = np.float32
    return int(_load().oracle_edge_sos(f(q[0]), f(q[1]), f(pi[0]), f(pi[1]), f(pj[0]), f(pj[1])))


def plane_sos(q, a, b, c) -> int:
    arrs = [np.ascontiguousarray(x, dtype=np.float32) for x in (q, a, b, c)]
    return int(_load().oracle_plane_sos(*[_p(x) for x in arrs]))


def tri_crossing(q, a, b, c) -> int:
    arrs = [np.ascontiguousarray(x, dtype=np.float32) for x in (q, a, b, c)]
    return int(_load().oracle_tri_crossing(*[_p(x) for x in arrs]))


def triangle_area(a, b, c, q) -> float:
    """Signed solid angle of one triangle seen from q (VOS, FP64)."""
    arrs = [np.ascontiguousarray(x, dtype=np.float32) for x in (a, b, c, q)]
    return float(_load().oracle_triangle_area(*[_p(x) for x in arrs]))


def reference(V, F, Q, with_direct: bool = False, quantize_bits: int = 0):
    """Everything the parity tests compare against, for one mesh and query set.

    Returns a dict with chi (int32), edges (oriented boundary), w_antipodal
    (float64), flags, and optionally w_direct (float64)."""
    c = chi(V, F, Q, quantize_bits)
    E = boundary(F, np.asarray(V).shape[0])
    w, fl = antipodal(V, E, Q, c, quantize_bits)
    out = {"chi": c, "edges": E, "w_antipodal": w, "flags": fl}
    if with_direct:
        out["w_direct"] = direct(V, F, Q)
    return out
