"""The CUDA paths against the closed-form fixtures of tests/golden/closed_forms.json
(derived by hand, see the file): antipodal w, direct sum, crossing count and
label of each mesh case; w of the parametric patch case.  FP32 outputs:
|dw| <= 2e-7 (a few units of rounding of w's magnitude, at most 1)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))
TOL = 2e-7


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


@pytest.mark.parametrize("m", GOLDEN["meshes"], ids=lambda m: m["name"])
def test_mesh_cases(gwn, m):
    for c in m["cases"]:
        V = np.asarray(m["V"], np.float32)
        F = np.asarray(m["F"], np.int32)
        if c.get("reverse"):
            F = F[:, ::-1].copy()
        q = torch.tensor([c["q"]], dtype=torch.float32, device="cuda")
        want = float(Fraction(c["w"]))
        with gwn.Mesh(V, F) as mesh:
            w, chi = mesh.query(q)
            wd = mesh.direct(q)
            lab = mesh.classify(q)
        assert abs(float(w[0]) - want) <= TOL, (m["name"], float(w[0]), want)
        assert abs(float(wd[0]) - want) <= TOL, (m["name"], float(wd[0]), want)
        assert int(lab[0]) == (1 if want > 0.5 else 0)


@pytest.mark.parametrize("p", GOLDEN["patches"], ids=lambda p: p["name"])
def test_patch_cases(gwn, p):
    a, b = p["a"], p["b"]
    C = np.zeros((1, 4, 4, 3), np.float32)
    for i in range(4):
        for j in range(4):
            C[0, i, j] = [-a + 2 * a * i / 3.0, -b + 2 * b * j / 3.0, 0.0]
    for fp64 in (0, 1):
        with gwn.ParamSurface(C, fp64=fp64) as s:
            for c in p["cases"]:
                w, chi = s.query(torch.tensor([c["q"]], dtype=torch.float32, device="cuda"))
                assert abs(float(w[0]) - float(Fraction(c["w"]))) <= TOL, (fp64, float(w[0]))
