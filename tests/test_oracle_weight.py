"""Pins of the oracle's weighted integral int h(f, g) w dt (no GPU).

The weight is a non-negative PCF (the weighted L_p distance of Sec. 2.2, the
weight multiplying |f - g|^p; the same weight on the inner product).  The
oracle's three-list rectangle iteration is checked against things other
than itself: the unweighted walk (w = 1, bit for bit), exact scaling by a
constant weight, the bounded integral for an indicator weight, closed forms
of indicator functions, linearity in w, the tail rule, an independent
union-grid evaluation and exact rational arithmetic.
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_07183_gb300 import synth

METRICS = [("l1", 1.0), ("l2", 2.0), ("lp", 3.0), ("gram", 1.0)]


def _random_weight(rng, n, t_max, compact=False):
    t = np.concatenate([[0.0], np.sort(rng.uniform(0, t_max, n - 1))])
    v = rng.uniform(0, 2, n)
    v[rng.random(n) < 0.3] = 0.0               # zero-weight stretches
    if compact:
        v[-1] = 0.0
    return t, v


def _dyadic_weight(rng, n):
    t = np.concatenate([[0.0], np.cumsum(rng.integers(1, 6, n - 1)).astype(float)])
    return t, rng.integers(0, 4, n).astype(float)


@pytest.mark.parametrize("metric,p", METRICS)
def test_unit_weight_is_the_unweighted_walk(metric, p):
    s = synth.random_set(30, seed=401, min_len=1, max_len=40)
    one = (np.array([0.0]), np.array([1.0]))
    for i in range(s.n):
        for j in range(s.n):
            a = oracle.integral_w(*s.pcf(i), *s.pcf(j), *one, metric, p)
            b = oracle.integral(*s.pcf(i), *s.pcf(j), metric, p)
            assert a == b or (np.isinf(a) and a == b)


@pytest.mark.parametrize("metric,p", METRICS)
def test_constant_weight_scales_exactly(metric, p):
    s = synth.dyadic(20, seed=402, max_len=20)
    for c in (0.0, 0.5, 2.0, 3.0):
        w = (np.array([0.0]), np.array([c]))
        for i in range(s.n):
            for j in range(i, s.n):
                a = oracle.integral_w(*s.pcf(i), *s.pcf(j), *w, metric, p)
                b = oracle.integral(*s.pcf(i), *s.pcf(j), metric, p)
                assert a == c * b


@pytest.mark.parametrize("metric,p", METRICS)
def test_indicator_weight_is_the_bounded_integral(metric, p):
    s = synth.dyadic(16, seed=403, max_len=25, final_zero=False)
    for a, b in ((3.0, 17.0), (0.0, 9.0), (11.0, 12.0)):
        w = (np.array([0.0, a, b]) if a > 0 else np.array([0.0, b]),
             np.array([0.0, 1.0, 0.0]) if a > 0 else np.array([1.0, 0.0]))
        for i in range(s.n):
            for j in range(s.n):
                x = oracle.integral_w(*s.pcf(i), *s.pcf(j), *w, metric, p)
                y = oracle.integral_ab(*s.pcf(i), *s.pcf(j), metric, p, a, b)
                assert x == y


@pytest.mark.parametrize("p", [1.0, 2.0, 3.5])
def test_indicator_closed_form(p):
    """f = c 1[a1, b1), g = 0, w = d 1[a2, b2): |c|^p d |[a1, b1) n [a2, b2)|."""
    rng = np.random.default_rng(404)
    for _ in range(200):
        a1, b1, a2, b2 = (float(x) for x in np.sort(rng.uniform(0.1, 10, 4))[rng.permutation(4)])
        a1, b1 = min(a1, b1), max(a1, b1)
        a2, b2 = min(a2, b2), max(a2, b2)
        c, d = rng.normal(), rng.uniform(0.1, 3)
        f = (np.array([0.0, a1, b1]), np.array([0.0, c, 0.0]))
        g = (np.array([0.0]), np.array([0.0]))
        w = (np.array([0.0, a2, b2]), np.array([0.0, d, 0.0]))
        ov = max(0.0, min(b1, b2) - max(a1, a2))
        got = oracle.integral_w(*f, *g, *w, "lp", p)
        assert abs(got - abs(c) ** p * d * ov) <= 1e-12 * max(1.0, abs(c) ** p * d * 10)


@pytest.mark.parametrize("metric,p", METRICS)
def test_linear_in_the_weight(metric, p):
    """int h (w1 + w2) = int h w1 + int h w2, exactly on dyadic inputs."""
    rng = np.random.default_rng(405)
    s = synth.dyadic(12, seed=406, max_len=20)
    for _ in range(10):
        w1, w2 = _dyadic_weight(rng, 6), _dyadic_weight(rng, 5)
        grid = np.union1d(w1[0], w2[0])
        w12 = (grid, brute.evaluate(*w1, grid) + brute.evaluate(*w2, grid))
        for i in range(s.n):
            for j in range(s.n):
                a = oracle.integral_w(*s.pcf(i), *s.pcf(j), *w12, metric, p)
                b = (oracle.integral_w(*s.pcf(i), *s.pcf(j), *w1, metric, p) +
                     oracle.integral_w(*s.pcf(i), *s.pcf(j), *w2, metric, p))
                assert a == b or (np.isinf(a) and np.isinf(b))


def test_tail_rule():
    """Unequal tails integrate to +-inf unless the weight vanishes there."""
    f = (np.array([0.0, 1.0]), np.array([2.0, 1.0]))
    g = (np.array([0.0, 2.0]), np.array([0.0, -1.0]))
    compact = (np.array([0.0, 3.0]), np.array([1.0, 0.0]))
    lasting = (np.array([0.0, 3.0]), np.array([0.0, 0.5]))
    assert oracle.integral_w(*f, *g, *compact, "l1") == 2.0 * 1 + 1.0 * 1 + 2.0 * 1
    assert oracle.integral_w(*f, *g, *lasting, "l1") == np.inf
    assert oracle.integral_w(*f, *g, *lasting, "gram") == -np.inf
    assert oracle.integral_w(*f, *f, *lasting, "l2") == 0.0


@pytest.mark.parametrize("metric,p", METRICS + [("lp", 2.5)])
def test_against_the_union_grid(metric, p):
    rng = np.random.default_rng(407)
    s = synth.random_set(14, seed=408, min_len=1, max_len=30)
    for k in range(6):
        w = _random_weight(rng, 12, 30.0, compact=k % 2 == 0)
        for i in range(s.n):
            for j in range(s.n):
                a = oracle.integral_w(*s.pcf(i), *s.pcf(j), *w, metric, p)
                b = brute.integral_w(*s.pcf(i), *s.pcf(j), *w, metric, p)
                if np.isinf(b):
                    assert a == b
                else:
                    assert abs(a - b) <= 1e-12 * max(1.0, abs(b))


@pytest.mark.parametrize("metric,p", [("l1", 1), ("l2", 2), ("lp", 3), ("gram", 1)])
def test_exact_rational(metric, p):
    rng = np.random.default_rng(409)
    s = synth.dyadic(8, seed=410, max_len=12, final_zero=False)
    for _ in range(4):
        w = _dyadic_weight(rng, 5)
        w[1][-1] = 0.0
        for i in range(s.n):
            for j in range(s.n):
                a = oracle.integral_w(*s.pcf(i), *s.pcf(j), *w, metric, p)
                e = brute.exact_integral_w(*s.pcf(i), *s.pcf(j), *w, metric, p)
                assert e is not None and a == float(e)
