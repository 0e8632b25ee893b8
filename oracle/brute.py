"""Second, independent oracle -- TEST INFRASTRUCTURE ONLY.

The integral of Eq. simpleint (Sec. 3) written the most direct way: build the
common refinement s_0 < ... < s_m of the two breakpoint sets explicitly
(union of the sets, Sec. 2), look up f(s_k) and g(s_k) by binary search, and
sum h(f(s_k), g(s_k)) (s_{k+1} - s_k).  The last cell [s_m, inf) adds 0 when
h is 0 there and +-inf otherwise.

``exact_integral`` does the same in rational arithmetic (fractions.Fraction)
for tiny inputs with integer exponent p, so its result is the exact value of
the integral of the given (float) inputs.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _h(metric, p, a, b):
    if metric == "l1":
        return np.abs(a - b)
    if metric == "l2":
        return (a - b) ** 2
    if metric == "lp":
        return np.abs(a - b) ** p
    if metric == "gram":
        return a * b
    raise ValueError(metric)


def union_grid(tf, tg):
    return np.unique(np.concatenate([np.asarray(tf, np.float64),
                                     np.asarray(tg, np.float64)]))


def evaluate(t, v, s):
    """Right-continuous PCF value at the points s."""
    idx = np.searchsorted(np.asarray(t, np.float64), s, side="right") - 1
    return np.asarray(v, np.float64)[idx]


def integral(tf, vf, tg, vg, metric="l1", p=1.0) -> float:
    s = union_grid(tf, tg)
    a = evaluate(tf, vf, s)
    b = evaluate(tg, vg, s)
    h = _h(metric, p, a, b)
    body = float(np.sum(h[:-1] * np.diff(s)))
    tail = h[-1]
    if tail != 0:
        return body + float(tail) * np.inf
    return body


def root(metric, p, x):
    if metric == "gram":
        return x
    e = {"l1": 1.0, "l2": 2.0}.get(metric, p)
    return x ** (1.0 / e)


def matrix(a, b=None, metric="l1", p=1.0, apply_root=True):
    bb = a if b is None else b
    out = np.empty((a.n, bb.n))
    for i in range(a.n):
        tf, vf = a.pcf(i)
        for j in range(bb.n):
            tg, vg = bb.pcf(j)
            I = integral(tf, vf, tg, vg, metric, p)
            out[i, j] = root(metric, p, I) if apply_root else I
    return out


def exact_integral(tf, vf, tg, vg, metric="l1", p=1):
    """Exact rational value (None if it diverges); p must be an integer."""
    tf = [Fraction(float(x)) for x in tf]
    tg = [Fraction(float(x)) for x in tg]
    vf = [Fraction(float(x)) for x in vf]
    vg = [Fraction(float(x)) for x in vg]
    grid = sorted(set(tf) | set(tg))

    def at(t, v, s):
        k = 0
        while k + 1 < len(t) and t[k + 1] <= s:
            k += 1
        return v[k]

    def h(x, y):
        if metric == "gram":
            return x * y
        d = abs(x - y)
        e = {"l1": 1, "l2": 2}.get(metric, p)
        return d ** int(e)

    total = Fraction(0)
    for k, s in enumerate(grid):
        val = h(at(tf, vf, s), at(tg, vg, s))
        if k + 1 < len(grid):
            total += val * (grid[k + 1] - s)
        elif val != 0:
            return None
    return total


def integral_w(tf, vf, tg, vg, tw, vw, metric="l1", p=1.0) -> float:
    """int h(f, g) w dt on the common refinement of the three breakpoint sets:
    every cell [s_k, s_{k+1}) adds h(f(s_k), g(s_k)) w(s_k) (s_{k+1} - s_k);
    the last cell adds 0 when h w = 0 there and +-inf otherwise."""
    s = np.unique(np.concatenate([np.asarray(x, np.float64) for x in (tf, tg, tw)]))
    hw = _h(metric, p, evaluate(tf, vf, s), evaluate(tg, vg, s)) * evaluate(tw, vw, s)
    body = float(np.sum(hw[:-1] * np.diff(s)))
    if hw[-1] != 0:
        return body + float(hw[-1]) * np.inf
    return body


def exact_integral_w(tf, vf, tg, vg, tw, vw, metric="l1", p=1):
    """Exact rational value of the weighted integral (None if it diverges)."""
    T = [[Fraction(float(x)) for x in a] for a in (tf, tg, tw)]
    V = [[Fraction(float(x)) for x in a] for a in (vf, vg, vw)]
    grid = sorted(set(T[0]) | set(T[1]) | set(T[2]))

    def at(t, v, s):
        k = 0
        while k + 1 < len(t) and t[k + 1] <= s:
            k += 1
        return v[k]

    e = {"l1": 1, "l2": 2}.get(metric, p)
    total = Fraction(0)
    for k, s in enumerate(grid):
        x, y, w = (at(T[q], V[q], s) for q in range(3))
        val = (x * y if metric == "gram" else abs(x - y) ** int(e)) * w
        if k + 1 < len(grid):
            total += val * (grid[k + 1] - s)
        elif val != 0:
            return None
    return total
