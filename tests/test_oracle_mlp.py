"""Pins of the float64 surrogate reference (oracle/mlp.py) to facts other than itself.

* Gradient: central finite differences of the loss, on every parameter block
  (a dropped ReLU mask, a transposed W_l or a missing 1/n fails here).
* Features: closed forms at the box centre (all sines 0, cosines 1) and at
  the low corner (x = -1: sin(-pi s) and cos(pi s) for s = 2^(7k/15); s_0 = 1,
  s_15 = 128 give sin 0 and cos -1, +1).
* Forward: the zero network returns b_5; a hand-wired path W_1[0][0] = 1,
  W_l[0][0] = 1, w_5[0] = 1 returns relu(x_0); a path that routes feature 1
  (x_1) through hidden unit 3 detects any transposed weight matrix.
* Adam: the first bias-corrected step moves each parameter by lr * g / (|g| + eps).
"""
import numpy as np
import pytest

from oracle import mlp


def _random_params(rng, scale=0.3):
    P = {}
    for name, shape in mlp._SHAPES:
        P[name] = rng.normal(scale=scale, size=shape)
    return mlp.pack(P)


def test_param_count():
    assert mlp.N_PARAMS == 64 * 128 + 64 + 3 * (64 * 64 + 64) + 64 + 1 == 20801


def test_features_centre_and_corner():
    box = np.array([-2.0, 0.0, 1.0, 2.0, 4.0, 3.0])
    centre = np.array([[0.0, 2.0, 2.0]])
    f = mlp.features(centre, box)[0]
    assert np.allclose(f[:3], 0.0, atol=1e-15)
    assert np.allclose(f[3:99:2], 0.0, atol=1e-12)     # sines
    assert np.allclose(f[4:99:2], 1.0, atol=1e-12)     # cosines
    assert np.all(f[99:] == 0.0)
    lo = np.array([[-2.0, 0.0, 1.0]])
    f = mlp.features(lo, box)[0]
    assert np.allclose(f[:3], -1.0)
    for d in range(3):
        assert abs(f[3 + 2 * d]) < 1e-12 and abs(f[4 + 2 * d] + 1.0) < 1e-12        # s_0 = 1
        assert abs(f[3 + 90 + 2 * d]) < 1e-9 and abs(f[4 + 90 + 2 * d] - 1.0) < 1e-12  # s_15 = 128
    # a middle frequency against its closed form: s_5 = 2^(7/3)
    s5 = 2.0 ** (7.0 / 3.0)
    assert abs(f[3 + 30] - np.sin(-np.pi * s5)) < 1e-12


def test_zero_network_returns_b5():
    P = {name: np.zeros(shape) for name, shape in mlp._SHAPES}
    P["b5"][0] = 0.375
    q = np.random.default_rng(0).uniform(-1, 1, size=(7, 3))
    y, _ = mlp.forward(mlp.pack(P), np.array([-1, -1, -1, 1, 1, 1.0]), q)
    assert np.all(y == 0.375)


def test_hand_wired_relu_path():
    P = {name: np.zeros(shape) for name, shape in mlp._SHAPES}
    P["W1"][0, 0] = 1.0
    for l in (2, 3, 4):
        P[f"W{l}"][0, 0] = 1.0
    P["w5"][0] = 1.0
    box = np.array([-1, -1, -1, 1, 1, 1.0])
    q = np.array([[0.25, 0.9, -0.3], [-0.5, 0.1, 0.2]])
    y, _ = mlp.forward(mlp.pack(P), box, q)
    assert np.allclose(y, [0.25, 0.0])


def test_transpose_probe():
    """x_1 enters hidden unit 3 (W_1[3][1]), moves 3 -> 5 -> 7 -> 11 (W_l[out][in]), read by w_5[11]."""
    P = {name: np.zeros(shape) for name, shape in mlp._SHAPES}
    P["W1"][3, 1] = 2.0
    P["W2"][5, 3] = 1.0
    P["W3"][7, 5] = 1.0
    P["W4"][11, 7] = 1.0
    P["w5"][11] = 1.0
    P["b2"][5] = 0.5
    box = np.array([-1, -1, -1, 1, 1, 1.0])
    q = np.array([[0.0, 0.3, 0.0], [0.0, -0.3, 0.0]])
    y, _ = mlp.forward(mlp.pack(P), box, q)
    assert np.allclose(y, [2 * 0.3 + 0.5, 0.5])


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = _random_params(rng)
    box = np.array([-1.5, -1.0, -0.5, 1.5, 1.0, 0.5])
    q = rng.uniform(box[:3], box[3:], size=(24, 3))
    t = rng.uniform(-0.5, 1.5, size=24)
    g, L = mlp.grad(p, box, q, t)
    assert abs(L - mlp.loss(p, box, q, t)) < 1e-14 * max(1.0, L)
    # a sample of coordinates in every block, plus the largest entries
    offsets, o = [], 0
    for name, shape in mlp._SHAPES:
        k = int(np.prod(shape))
        offsets += list(o + rng.choice(k, size=min(k, 12), replace=False))
        o += k
    offsets += list(np.argsort(-np.abs(g))[:10])
    h = 1e-6
    for i in offsets:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, box, q, t) - mlp.loss(p - e, box, q, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m1, v1 = mlp.adam_step(p, np.zeros(50), np.zeros(50), g, 1, lr=1e-3, eps=1e-8)
    assert np.allclose(p - p1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
