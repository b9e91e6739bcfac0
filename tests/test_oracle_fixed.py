"""Pins of the oracle's fixed-point predicates (Supp. S2.1: inputs snapped to a
30-bit grid, perturbed signs decided in integer arithmetic).

* On inputs that are multiples of the quantum (integer vertex and query
  coordinates with a power-of-two quantum), snapping is exact, so the
  fixed-point crossing counts and branch-cut signs must equal the exact-FP32
  ones on every query, including queries on vertices, edges and faces: the two
  implementations share no predicate code (bit-level expansions of the FP32
  values against 128-bit integers of the snapped ones).
* The quantum follows from the bounding box: half-extent 4 gives 2^-26, so a
  triangle 2^-30 above a query snaps onto the query's height (not counted),
  while one 2^-26 above stays above (counted) - the exact predicates count both.
* On float inputs a random query sits within a quantum of the surface with
  probability ~1e-8, so results agree with the exact predicates.
"""
import numpy as np

import gen
import oracle


def test_integer_inputs_match_exact_everywhere():
    mesh, Q, kinds = gen.precision_workload(n_query=6000)
    a = oracle.chi(mesh.V, mesh.F, Q)
    b = oracle.chi(mesh.V, mesh.F, Q, quantize_bits=30)
    assert np.array_equal(a, b)
    E = oracle.boundary(mesh.F, mesh.nv)
    wa, fa = oracle.antipodal(mesh.V, E, Q, a)
    wb, fb = oracle.antipodal(mesh.V, E, Q, b, quantize_bits=30)
    assert np.array_equal(fa, fb)
    assert np.array_equal(wa, wb)


def test_quantum_from_bounding_box():
    # a unit square in the plane z = h; two extra vertices fix the box to
    # x in [-3, 5], z in [-4, 4]: centre (1, 0, 0), half-extent 4, quantum 2^-26
    def mesh_at(h):
        V = np.array([[-1, -1, h], [1, -1, h], [1, 1, h], [-1, 1, h], [-3, 0, -4], [5, 0, 4]], np.float32)
        F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
        return V, F
    q = np.array([[0.25, 0.1, 0.0]], np.float32)
    V, F = mesh_at(2.0 ** -30)
    assert oracle.chi(V, F, q)[0] == 1
    assert oracle.chi(V, F, q, quantize_bits=30)[0] == 0     # snapped onto the query's height
    V, F = mesh_at(2.0 ** -26)
    assert oracle.chi(V, F, q)[0] == 1
    assert oracle.chi(V, F, q, quantize_bits=30)[0] == 1     # one quantum above: still above
    V, F = mesh_at(2.0 ** -27 * 1.5)                          # 0.75 quantum: rounds up to 1
    assert oracle.chi(V, F, q, quantize_bits=30)[0] == 1


def test_float_inputs_agree_with_exact():
    mesh, rng = gen.displaced_soup(3, seed=31)
    Q = np.concatenate([gen.queries_uniform_bbox(mesh.V, 1500, rng),
                        gen.queries_near_surface(mesh.V, mesh.F, 1500, rng)])
    a = oracle.chi(mesh.V, mesh.F, Q)
    b = oracle.chi(mesh.V, mesh.F, Q, quantize_bits=30)
    assert np.array_equal(a, b)
    E = oracle.boundary(mesh.F, mesh.nv)
    wa, _ = oracle.antipodal(mesh.V, E, Q, a)
    wb, _ = oracle.antipodal(mesh.V, E, Q, b, quantize_bits=30)
    assert np.array_equal(wa, wb)
