"""Float64 reference of the learned surrogate of w.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
may import this module; the library never does.

The paper has no network: its conclusion (Sec. 8, future work) names a fast
approximation of the fractional part of w as an open direction, and this
library adds one as an optional front end to the exact antipodal path.  The
network is therefore defined here, in plain numpy float64, exactly as the
library documents it:

    x_d   = 2 (q_d - lo_d) / (hi_d - lo_d) - 1                 d = 0, 1, 2
    f     = [x_0, x_1, x_2,
             sin(pi s_k x_d), cos(pi s_k x_d)  for k < 16, d < 3]  (feature
             3 + 6k + 2d is the sine, 4 + 6k + 2d the cosine), s_k = 2^(7k/15),
             then zeros up to width 128
    h_1   = relu(W_1 f + b_1)          W_1: [64][128]
    h_l   = relu(W_l h_{l-1} + b_l)    W_l: [64][64], l = 2, 3, 4
    w_hat = w_5 . h_4 + b_5
    L     = mean over the batch of (w_hat - t)^2

Parameter vector (float32 on the library side, float64 here), in order:
W_1 (row-major, 64 x 128), b_1, W_2, b_2, W_3, b_3, W_4, b_4 (64 x 64 and
64 each), w_5 (64), b_5 (1): 20801 numbers.

Adam (Kingma and Ba 2015, Algorithm 1): m <- b1 m + (1-b1) g,
v <- b2 v + (1-b2) g^2, p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Pins (tests/test_oracle_mlp.py): central finite differences of ``loss``
against ``grad``; closed-form features at the box centre and corners;
hand-wired networks whose output is known (a single path that computes
relu(x_0), the zero network giving b_5, a layer-order probe that fails if any
W_l is transposed); the first Adam step's closed form.
"""
from __future__ import annotations

import numpy as np

N_FREQ = 16
N_FEAT = 3 + 6 * N_FREQ     # 99
N_IN = 128
N_HID = 64

_SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
           ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_HID, N_HID)), ("b4", (N_HID,)),
           ("w5", (N_HID,)), ("b5", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in _SHAPES)   # 20801


def unpack(p) -> dict:
    """Flat parameter vector -> dict of float64 arrays (views are copied)."""
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    if p.size != N_PARAMS:
        raise ValueError(f"expected {N_PARAMS} parameters, got {p.size}")
    out, o = {}, 0
    for name, shape in _SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape).copy()
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in _SHAPES])


def frequencies() -> np.ndarray:
    """s_k = 2^(7k/15), k = 0..15 (log-spaced from 1 to 128)."""
    return np.array([2.0 ** (7.0 * k / 15.0) for k in range(N_FREQ)])


def normalise(q, box) -> np.ndarray:
    """Map the box [lo, hi] (box = lo xyz, hi xyz) to [-1, 1]^3."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, 3)
    lo = np.asarray(box[:3], dtype=np.float64)
    hi = np.asarray(box[3:], dtype=np.float64)
    return 2.0 * (q - lo) / (hi - lo) - 1.0


def features(q, box) -> np.ndarray:
    """[n, 128] Fourier features of the queries, zero-padded."""
    x = normalise(q, box)
    f = np.zeros((x.shape[0], N_IN))
    f[:, 0:3] = x
    s = frequencies()
    for k in range(N_FREQ):
        for d in range(3):
            f[:, 3 + 6 * k + 2 * d] = np.sin(np.pi * s[k] * x[:, d])
            f[:, 4 + 6 * k + 2 * d] = np.cos(np.pi * s[k] * x[:, d])
    return f


def forward(p, box, q):
    """w_hat [n] and the cache (features, pre-activations z_l, activations h_l)."""
    P = unpack(p)
    f = features(q, box)
    h = f
    zs, hs = [], []
    for l in range(1, 5):
        z = h @ P[f"W{l}"].T + P[f"b{l}"]
        h = np.maximum(z, 0.0)
        zs.append(z)
        hs.append(h)
    y = h @ P["w5"] + P["b5"][0]
    return y, {"f": f, "z": zs, "h": hs, "P": P}


def loss(p, box, q, t) -> float:
    y, _ = forward(p, box, q)
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    return float(np.mean((y - t) ** 2))


def grad(p, box, q, t):
    """(dL/dp as a flat vector, L) by reverse-mode differentiation of the chain above."""
    y, c = forward(p, box, q)
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    n = y.shape[0]
    P = c["P"]
    dy = 2.0 * (y - t) / n                        # dL/dw_hat
    G = {"w5": c["h"][3].T @ dy, "b5": np.array([dy.sum()])}
    delta = np.outer(dy, P["w5"]) * (c["z"][3] > 0)   # dL/dz_4
    for l in range(4, 0, -1):
        h_prev = c["f"] if l == 1 else c["h"][l - 2]
        G[f"W{l}"] = delta.T @ h_prev
        G[f"b{l}"] = delta.sum(axis=0)
        if l > 1:
            delta = (delta @ P[f"W{l}"]) * (c["z"][l - 2] > 0)
    return pack(G), float(np.mean((y - t) ** 2))


def adam_step(p, m, v, g, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at (1-based) step number ``step``; returns (p, m, v)."""
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return np.asarray(p, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v
