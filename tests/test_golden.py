"""Pins of the oracle to the closed-form fixtures of tests/golden/closed_forms.json.

Every value there is derived by hand (Girard's theorem of Sec. 3, the symmetry
of regular solids, the rectangle seen from its axis), independently of the
oracle and of the CUDA path; each fixture carries its derivation.  The
oracle's direct sum (Eq. 2 with the VOS area, Eq. 6), its antipodal w (Eq. 9
with exact crossing counts) and its parametric definition (Eq. 1 by adaptive
and by fixed quadrature) must reproduce them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))


def mesh_cases():
    for m in GOLDEN["meshes"]:
        for k, c in enumerate(m["cases"]):
            yield pytest.param(m, c, id=f"{m['name']}-{k}")


def golden_mesh(m, c):
    V = np.asarray(m["V"], np.float32)
    F = np.asarray(m["F"], np.int32)
    if c.get("reverse"):
        F = F[:, ::-1].copy()
    return V, F, np.asarray([c["q"]], np.float32), float(Fraction(c["w"]))


@pytest.mark.parametrize("m,c", list(mesh_cases()))
def test_direct_and_antipodal(m, c):
    V, F, Q, want = golden_mesh(m, c)
    wd = oracle.direct(V, F, Q)[0]
    assert abs(wd - want) <= 1e-12, (m["name"], wd, want)
    ref = oracle.reference(V, F, Q)
    assert ref["flags"][0] == 0
    assert abs(ref["w_antipodal"][0] - want) <= 1e-12, (m["name"], ref["w_antipodal"][0], want)


def bilinear_patch(a, b):
    C = np.zeros((4, 4, 3))
    for i in range(4):
        for j in range(4):
            C[i, j] = [-a + 2 * a * i / 3.0, -b + 2 * b * j / 3.0, 0.0]
    return C.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("p", GOLDEN["patches"], ids=lambda p: p["name"])
def test_parametric_definition(p):
    pytest.importorskip("scipy")
    from oracle import parametric as par
    C = bilinear_patch(p["a"], p["b"])
    for c in p["cases"]:
        want = float(Fraction(c["w"]))
        assert abs(par.w_direct([C], c["q"]) - want) <= 1e-8
        assert abs(par.w_gauss([C], c["q"], n_sub=16) - want) <= 1e-6
