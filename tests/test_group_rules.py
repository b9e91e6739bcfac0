"""The two group acceptance tests of the boundary kernel, checked as mathematics
in FP64 on random edge terms (no GPU): a term's angle is atan2(n, d) with
n = A_y B_x - A_x B_y and d = H_a H_b + A_x B_x + A_y B_y (H = 1 - A_z) for unit
vectors A, B from the query to the edge's ends (Eq. 9's antipodal term with
x1 = -z).  Under either test the argument of the running complex product of
the accepted terms' (d + i n) must equal the sum of their angles, and the
per-term test alone must fail that once its bound is dropped (the wrap it
prevents)."""
import numpy as np

TAN_GROUP, ACCEPT, MIN_D = 0.41, 2e-5, 5e-5


def _terms(rng, n, spread):
    """n, d of random edges: endpoints around the query at random distances,
    edge lengths `spread` times the distance (large spread: steep terms)."""
    c = rng.normal(size=(n, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    r = 10.0 ** rng.uniform(-1, 1, size=(n, 1))
    a = c * r + rng.normal(size=(n, 3)) * spread * r
    b = c * r + rng.normal(size=(n, 3)) * spread * r
    A = a / np.linalg.norm(a, axis=1, keepdims=True)
    B = b / np.linalg.norm(b, axis=1, keepdims=True)
    ha, hb = 1.0 - A[:, 2], 1.0 - B[:, 2]
    num = A[:, 1] * B[:, 0] - A[:, 0] * B[:, 1]
    den = ha * hb + A[:, 0] * B[:, 0] + A[:, 1] * B[:, 1]
    return num, den


def _group(num, den, accept):
    """The running product of one group: returns (its argument, the accepted angles' sum, accepted count)."""
    z = 1.0 + 0.0j
    total = 0.0
    k = 0
    for n, d in zip(num, den):
        cand = z * complex(d, n)
        if accept(n, d, cand):
            z = cand
            total += np.arctan2(n, d)
            k += 1
    return np.angle(z), total, k


def per_term(n, d, _):
    return TAN_GROUP * d - abs(n) > ACCEPT


def running(n, d, cand):
    return d > MIN_D and cand.real > 0.0


def test_angle_identity_for_both_tests():
    rng = np.random.default_rng(5)
    for spread in (0.05, 0.5, 3.0):
        num, den = _terms(rng, 8 * 4000, spread)
        acc = {"per_term": 0, "running": 0}
        for g in range(4000):
            sl = slice(8 * g, 8 * g + 8)
            for name, rule in (("per_term", per_term), ("running", running)):
                arg, total, k = _group(num[sl], den[sl], rule)
                assert abs(arg - total) < 1e-12, (spread, g, name, arg, total)
                acc[name] += k
        # the running test accepts at least as many of the steep terms
        assert acc["running"] >= acc["per_term"]
        if spread == 3.0:
            assert acc["running"] > 1.05 * acc["per_term"]


def test_running_product_stays_in_right_half_plane():
    rng = np.random.default_rng(6)
    num, den = _terms(rng, 16 * 2000, 2.0)
    for g in range(2000):
        z = 1.0 + 0.0j
        for n, d in zip(num[16 * g:16 * g + 16], den[16 * g:16 * g + 16]):
            cand = z * complex(d, n)
            if running(n, d, cand):
                z = cand
            assert z.real > 0.0 and abs(np.angle(z)) < np.pi / 2


def test_without_a_bound_the_product_wraps():
    """Accepting every term with d > 0 (angles below pi/2 each, no running
    test) lets 8 terms pass +-pi, where the product's argument is no longer the
    sum: the reason for either test."""
    rng = np.random.default_rng(7)
    num, den = _terms(rng, 8 * 4000, 3.0)
    wraps = 0
    for g in range(4000):
        arg, total, _ = _group(num[8 * g:8 * g + 8], den[8 * g:8 * g + 8], lambda n, d, c: d > 0.0)
        wraps += abs(arg - total) > 1e-9
    assert wraps > 0
