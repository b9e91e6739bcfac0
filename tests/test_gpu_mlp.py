"""GPU tests of the tensor-core (tcgen05) building blocks and the surrogate MLP."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwn():
    import paper_2605_01536_gb300 as g
    g.load()
    return g


@pytest.mark.parametrize("K", [64, 128])
def test_tc_gemm_selftest(gwn, K):
    """One tcgen05 BF16 MMA chain (128 x 64 x K, FP32 accumulators in TMEM)
    against a float64 product of the same BF16 values."""
    lib = gwn.load()
    rng = np.random.default_rng(K)
    A = torch.from_numpy(rng.normal(size=(128, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.from_numpy(rng.normal(size=(64, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    C = torch.empty((128, 64), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.gwn_debug_tc_gemm(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), K,
                               ctypes.c_void_p(C.data_ptr()), stream)
    assert rc == 0, lib.gwn_last_error()
    ref = A.float().cpu().double().numpy() @ B.float().cpu().double().numpy().T
    err = np.abs(C.cpu().numpy() - ref).max()
    assert err <= 1e-4 * np.abs(ref).max(), err


# ---------------------------------------------------------------------------
# Surrogate MLP against the float64 reference (oracle/mlp.py)
# ---------------------------------------------------------------------------
from oracle import mlp as ref  # noqa: E402

U = 2.0 ** -8          # unit roundoff of BF16 (8 significand bits, round to nearest)
U32 = 2.0 ** -24       # FP32
NSIG = 6.0             # tolerance in standard deviations of the modelled rounding error


def _params(rng):
    """Random parameters (He-scaled weights); W_1..W_4 are BF16-representable,
    so that the GPU's BF16 weight copies are exact and the only rounding left is
    per-sample (features and stored activations), which the model below treats
    as independent."""
    P = {}
    for name, shape in ref._SHAPES:
        if name.startswith("W"):
            w = rng.normal(scale=np.sqrt(2.0 / shape[1]), size=shape).astype(np.float32)
            P[name] = torch.from_numpy(w).to(torch.bfloat16).float().numpy()
        elif name == "w5":
            P[name] = rng.normal(scale=0.2, size=shape)
        else:
            P[name] = rng.normal(scale=0.05, size=shape)
    return ref.pack(P).astype(np.float32)


def _sigma(p, box, q, t=None):
    """Standard deviation of the GPU's deviation from the float64 network under a
    first-order probabilistic rounding-error model (each rounding an independent,
    zero-mean error; Higham and Mary, SIAM J. Sci. Comput. 2019).

    Roundings on the GPU: every feature is computed in FP32 (phase error
    pi s_k |x| 2^-23, plus 1e-6 for the SFU sine / cosine) and stored as BF16; every
    hidden activation and every backward delta is stored as BF16 (variance
    u^2 x^2 / 3); products accumulate in FP32.  Errors propagate linearly
    (squared weights, ReLU masks).  Where a pre-activation lies within
    NSIG sigma of zero the ReLU mask may differ; the forward error is then still
    bounded by the pre-activation's (ReLU is 1-Lipschitz), and the backward
    delta of that unit is given the whole unmasked gradient as its sigma.
    Returns (sigma of w_hat, sigma of the gradient vector, sigma of the loss).
    """
    y, c = ref.forward(p.astype(np.float64), box, q)
    P, f = c["P"], c["f"]
    x = np.abs(ref.normalise(q, box))
    s = ref.frequencies()
    Vf = U * U * f * f / 3.0
    for k in range(ref.N_FREQ):
        for d in range(3):
            # FP32 phase error of the argument, plus the SFU sine / cosine of the
            # reduced argument (absolute error below 1e-6)
            ph = (np.pi * s[k] * (x[:, d] + 1.0) * 2 * U32) ** 2 + (1e-6) ** 2
            Vf[:, 3 + 6 * k + 2 * d] += ph
            Vf[:, 4 + 6 * k + 2 * d] += ph
    Vh, h = Vf, f
    Vz, Vh32, Vhb = [], [], []
    for l in range(1, 5):
        W2 = P[f"W{l}"] ** 2
        vz = Vh @ W2.T + h.shape[1] * (U32 ** 2) * ((h * h) @ W2.T)
        z = c["z"][l - 1]
        live = z > -NSIG * np.sqrt(vz)
        vh32 = vz * live
        hl = c["h"][l - 1]
        vhb = vh32 + U * U * hl * hl / 3.0
        Vz.append(vz), Vh32.append(vh32), Vhb.append(vhb)
        Vh, h = vhb, hl
    h4 = c["h"][3]
    Vy = Vh32[3] @ (P["w5"] ** 2) + 64 * U32 ** 2 * ((h4 * h4) @ (P["w5"] ** 2))
    if t is None:
        return np.sqrt(Vy), None, None
    n = len(y)
    e = y - np.asarray(t, np.float64)
    dy = 2 * e / n
    Vdy = 4 * Vy / n ** 2
    G = {"w5": (h4 * h4).T @ Vdy + (dy * dy) @ Vh32[3], "b5": np.array([Vdy.sum()])}
    g = np.outer(dy, P["w5"])
    Vg = np.outer(Vdy, P["w5"] ** 2)
    for l in range(4, 0, -1):
        z = c["z"][l - 1]
        unsure = np.abs(z) <= NSIG * np.sqrt(Vz[l - 1])
        d = g * (z > 0)
        Vd = np.where(unsure, g * g + Vg, Vg * (z > 0)) + U * U * d * d / 3.0
        hp = f if l == 1 else c["h"][l - 2]
        Vhp = Vf if l == 1 else Vhb[l - 2]
        G[f"W{l}"] = Vd.T @ (hp * hp) + (d * d).T @ Vhp + n * U32 ** 2 * ((d * d).T @ (hp * hp))
        G[f"b{l}"] = Vd.sum(0) + n * U32 ** 2 * (d * d).sum(0)
        if l > 1:
            W = P[f"W{l}"]
            g = d @ W
            Vg = Vd @ (W * W) + 64 * U32 ** 2 * ((d * d) @ (W * W))
    VL = (4 * e * e * Vy).sum() / n ** 2
    return np.sqrt(Vy), np.sqrt(ref.pack(G)), float(np.sqrt(VL))


def _box_and_queries(rng, n):
    box = np.array([-1.2, -0.8, -1.0, 1.3, 0.9, 1.1], np.float32)
    q = rng.uniform(box[:3], box[3:], size=(n, 3)).astype(np.float32)
    return box, q


@pytest.fixture(scope="module")
def tiny_mesh(gwn):
    import gen
    m = gen.small_cap(3, 0.8)
    mesh = gwn.Mesh(m.V, m.F)
    yield mesh
    mesh.close()


@pytest.mark.parametrize("n", [1, 127, 1000, 4133])
def test_surrogate_forward_matches_reference(gwn, tiny_mesh, n):
    rng = np.random.default_rng(100 + n)
    p = _params(rng)
    box, q = _box_and_queries(rng, n)
    tiny_mesh.set_surrogate_params(p, box)
    got = tiny_mesh.surrogate_predict(torch.from_numpy(q).cuda()).cpu().numpy().astype(np.float64)
    want, _ = ref.forward(p.astype(np.float64), box.astype(np.float64), q)
    sy, _, _ = _sigma(p, box.astype(np.float64), q)
    assert np.all(np.abs(got - want) <= NSIG * sy + 1e-7), np.max(np.abs(got - want) / sy)
    # the tolerance is not vacuous: it stays well below the spread of the outputs
    assert np.median(NSIG * sy) < 0.1 * max(np.std(want), 1e-3) or n == 1


def test_surrogate_params_roundtrip(gwn, tiny_mesh):
    rng = np.random.default_rng(5)
    p = _params(rng)
    box = np.array([-1, -2, -3, 1, 2, 3], np.float32)
    tiny_mesh.set_surrogate_params(p, box)
    p2, box2 = tiny_mesh.surrogate_params()
    assert np.array_equal(p, p2) and np.array_equal(box, box2)


@pytest.mark.parametrize("n", [300, 2600])
def test_surrogate_gradient_matches_reference(gwn, tiny_mesh, n):
    """One forward + backward on the tensor cores against the float64 gradient;
    n = 2600 spans three weight-gradient CTAs (1024 rows each) and a ragged
    128-row chunk."""
    rng = np.random.default_rng(200 + n)
    p = _params(rng)
    box, q = _box_and_queries(rng, n)
    t = rng.uniform(-0.2, 1.2, size=n).astype(np.float32)
    tiny_mesh.set_surrogate_params(p, box)
    g, L = tiny_mesh.surrogate_grad(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda())
    g_ref, L_ref = ref.grad(p.astype(np.float64), box.astype(np.float64), q, t)
    _, sg, sL = _sigma(p, box.astype(np.float64), q, t)
    assert abs(L - L_ref) <= NSIG * sL + 1e-6 * L_ref, (L, L_ref, sL)
    bad = np.abs(g - g_ref) > NSIG * sg + 1e-6 * np.abs(g_ref) + 1e-9
    assert not bad.any(), (np.flatnonzero(bad)[:10], (np.abs(g - g_ref) / (sg + 1e-30))[bad][:10])
    # the whole vector: sum of squared errors against its modelled expectation (a
    # sum of many independent terms concentrates near its mean; 3x leaves room)
    err = np.linalg.norm(g - g_ref)
    assert err <= 3.0 * np.linalg.norm(sg), (err, np.linalg.norm(sg), np.linalg.norm(g_ref))


@pytest.mark.parametrize("level,res", [(4, 48), (6, 96)])
def test_surrogate_train_classify_gain(gwn, level, res):
    """Training lowers the loss and is bit-reproducible (gradients summed in
    fixed point); with the surrogate attached, classify answers most queries
    from the network and sends the rest (|w_hat - 1/2| <= margin, inside the
    surface band, or w_hat farther than 0.25 from the exact crossing count)
    through the exact path, whose answers match the plain classify.  After
    fallback there is no label error on any cell of the grid, at the default
    margin and at the margin calibrated on held-out samples."""
    import gen
    m, S, G = gen.surrogate_workload(level=level, n_train=200_000, res=res, seed=4)
    with gwn.Mesh(m.V, m.F) as mesh:
        qg = torch.from_numpy(G).cuda()
        lab_exact, w_exact = mesh.classify(qg, want_w=True)
        lab_exact, w_exact = lab_exact.cpu().numpy(), w_exact.cpu().numpy()
        s = torch.from_numpy(S).cuda()
        loss_short = mesh.train_surrogate(s, config={"steps": 20, "seed": 7})
        loss = mesh.train_surrogate(s, config={"steps": 3000, "seed": 7})
        params = mesh.surrogate_params()[0].copy()
        # half the samples lie within ~1e-3 of the surface, where w jumps by 1: the
        # loss cannot go near zero, but training must cut it well down
        assert loss < 0.5 * loss_short, (loss_short, loss)
        # the same seed and samples give the same network, bit for bit
        assert mesh.train_surrogate(s, config={"steps": 3000, "seed": 7}) == loss
        assert np.array_equal(mesh.surrogate_params()[0], params)
        w_hat = mesh.surrogate_predict(qg).cpu().numpy()
        chi = mesh.chi(qg).cpu().numpy()

        def run(margin):
            mesh.counters(reset=True)
            lab, w = mesh.classify(qg, want_w=True)
            lab, w = lab.cpu().numpy(), w.cpu().numpy()
            c = mesh.counters()
            answered = (w == w_hat) & (np.abs(w_hat - 0.5) > margin)
            assert c["surrogate_queries"] == len(G)
            assert c["surrogate_queries"] - c["surrogate_fallbacks"] == int(answered.sum())
            fb = ~answered
            # fallback queries: the exact path's labels, w within the parity tolerance
            assert np.array_equal(lab[fb], lab_exact[fb])
            assert np.max(np.abs(w[fb] - w_exact[fb]), initial=0.0) <= 1e-5
            # network answers: the label is w_hat's side of 1/2, and w_hat agrees with chi
            assert np.array_equal(lab[answered], (w_hat[answered] > 0.5).astype(np.uint8))
            assert np.all(np.abs(w_hat[answered] - chi[answered]) <= 0.25)
            return float(answered.mean()), int((lab != lab_exact).sum())

        answered, errors = run(0.1)
        print(f"surrogate level {level}, {res}^3: answered {answered:.3f}, label errors {errors} of {len(G)}, "
              f"loss {loss:.2e}")
        assert answered > 0.7
        assert errors == 0
        # calibrated gate: the margin at which no held-out sample (drawn like the grid) is
        # answered with a wrong label
        rng = np.random.default_rng(11)
        lo, hi = G.min(0), G.max(0)
        held = torch.from_numpy(rng.uniform(lo, hi, size=(400_000, 3)).astype(np.float32)).cuda()
        margin, held_err = mesh.calibrate_surrogate(held, max_error_rate=0.0, min_margin=0.1)
        assert 0.1 <= margin and held_err == 0
        answered_c, errors_c = run(margin)
        print(f"surrogate, calibrated margin {margin:.4f}: answered {answered_c:.3f}, label errors {errors_c}")
        assert errors_c == 0
        assert answered_c > 0.5
        mesh.detach_surrogate()
        lab2 = mesh.classify(qg).cpu().numpy()
        assert np.array_equal(lab2, lab_exact)


def test_surrogate_save_load(gwn, tmp_path):
    import gen
    m = gen.small_cap(3, 0.8)
    rng = np.random.default_rng(9)
    box, q = _box_and_queries(rng, 777)
    qd = torch.from_numpy(q).cuda()
    with gwn.Mesh(m.V, m.F) as a, gwn.Mesh(m.V, m.F) as b:
        a.train_surrogate(qd, config={"steps": 30, "batch": 512, "seed": 3})
        path = str(tmp_path / "sur.bin")
        a.save_surrogate(path)
        b.load_surrogate(path)
        assert np.array_equal(a.surrogate_params()[0], b.surrogate_params()[0])
        assert torch.equal(a.surrogate_predict(qd), b.surrogate_predict(qd))
        with open(path, "r+b") as fh:
            fh.write(b"XXXX")
        with pytest.raises(gwn.GwnError):
            b.load_surrogate(path)


def test_surrogate_gate_without_chi_test(gwn):
    """chi_tol < 0 switches the crossing-count test off: the gate is margin and
    band only, the fallback computes its own crossing counts, and its labels
    are the exact path's."""
    import gen
    m, S, G = gen.surrogate_workload(level=3, n_train=50_000, res=24, seed=4)
    with gwn.Mesh(m.V, m.F) as mesh:
        qg = torch.from_numpy(G).cuda()
        lab_exact = mesh.classify(qg).cpu().numpy()
        mesh.train_surrogate(torch.from_numpy(S).cuda(), config={"steps": 300, "seed": 7, "chi_tol": -1.0})
        w_hat = mesh.surrogate_predict(qg).cpu().numpy()
        lab, w = mesh.classify(qg, want_w=True)
        lab, w = lab.cpu().numpy(), w.cpu().numpy()
        answered = (w == w_hat) & (np.abs(w_hat - 0.5) > 0.1)
        assert np.array_equal(lab[~answered], lab_exact[~answered])
        assert np.array_equal(lab[answered], (w_hat[answered] > 0.5).astype(np.uint8))
        assert answered.any()
