"""Pins for the CPU oracle (runs without a GPU).

Each test ties the oracle to something other than itself: numbers printed in
the paper, closed forms, invariants of the definition, an independent union-
grid implementation, and exact rational arithmetic.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_07183_gb300 import synth

from conftest import read_golden


def _pcf(rows):
    rows = np.asarray(rows, dtype=np.float64)
    return rows[:, 0].copy(), rows[:, 1].copy()


def _set_from_pcfs(pcfs):
    offs = np.zeros(len(pcfs) + 1, np.int64)
    offs[1:] = np.cumsum([len(t) for t, _ in pcfs])
    t = np.concatenate([t for t, _ in pcfs])
    v = np.concatenate([v for _, v in pcfs])
    return synth.PcfSet(offs, t, v)


# --------------------------------------------------------------------------
# Values printed in the paper
# --------------------------------------------------------------------------
def test_worked_example_sec5_2():
    """Sec. 5.2: pdist (L1), pdist p=3.5 and l2_kernel of f1..f4."""
    g = read_golden("worked_example_sec5_2.txt")
    pcfs = [_pcf(g[f"pcf f{i}"]) for i in range(1, 5)]
    X = _set_from_pcfs(pcfs)
    l1 = oracle.matrix(X, metric="l1")
    np.testing.assert_array_equal(l1, g["matrix l1 p=1"])
    gram = oracle.matrix(X, metric="gram")
    np.testing.assert_array_equal(gram, g["matrix gram p=1"])
    l35 = oracle.matrix(X, metric="lp", p=3.5)
    np.testing.assert_allclose(l35, g["matrix lp p=3.5"], rtol=0, atol=6e-9)
    assert np.all(np.diag(l35) == 0.0)


def test_figure1_rectangles():
    """Sec. 3, Figure 1: the rectangle sequence of Alg. 1."""
    g = read_golden("figure1_rectangles.txt")
    tf, vf = _pcf(g["pcf f"])
    tg, vg = _pcf(g["pcf g"])
    rects = oracle.rectangles(tf, vf, tg, vg)
    np.testing.assert_array_equal(rects, g["rectangles"])
    # integral of Alg. 2 over these rectangles, L1: 2*2 + 1*1 + 1*1 + 1*1 = 7
    assert oracle.integral(tf, vf, tg, vg, "l1") == 7.0


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------
def _indicator(c, a, b):
    """c * 1_[a, b) as a PCF (t_0 = 0)."""
    if a == 0.0:
        return np.array([0.0, b]), np.array([c, 0.0])
    return np.array([0.0, a, b]), np.array([0.0, c, 0.0])


@pytest.mark.parametrize("seed", range(20))
def test_indicator_overlap_closed_form(seed):
    rng = np.random.default_rng(seed)
    a, b = np.sort(rng.uniform(0, 10, 2))
    a2, b2 = np.sort(rng.uniform(0, 10, 2))
    if seed % 5 == 0:
        a = 0.0
    c, d = rng.normal(size=2) * 3
    tf, vf = _indicator(c, a, b)
    tg, vg = _indicator(d, a2, b2)
    ov = max(0.0, min(b, b2) - max(a, a2))
    assert oracle.integral(tf, vf, tg, vg, "gram") == pytest.approx(c * d * ov, rel=1e-13, abs=1e-13)
    for metric, p in (("l1", 1.0), ("l2", 2.0), ("lp", 3.0), ("lp", 3.5)):
        want = (abs(c) ** p * (b - a) + abs(d) ** p * (b2 - a2)
                - ov * (abs(c) ** p + abs(d) ** p - abs(c - d) ** p))
        got = oracle.integral(tf, vf, tg, vg, metric, p)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12), (metric, p)


def test_self_distance_exactly_zero_and_norm():
    s = synth.random_set(30, seed=3, max_len=50)
    for i in range(s.n):
        t, v = s.pcf(i)
        for metric, p in (("l1", 1), ("l2", 2), ("lp", 3.5)):
            assert oracle.integral(t, v, t, v, metric, p) == 0.0
        # <f, f> = sum v_k^2 dt_k (segment iteration, Alg. 3)
        want = float(np.sum(v[:-1] ** 2 * np.diff(t)))
        assert oracle.integral(t, v, t, v, "gram") == pytest.approx(want, rel=1e-14)
        assert oracle.segment_sq(t, v) == pytest.approx(want, rel=1e-14)


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("metric,p", [("l1", 1), ("l2", 2), ("lp", 3.5), ("gram", 1)])
def test_symmetry_bitwise(metric, p):
    s = synth.random_set(25, seed=11, max_len=60)
    M = oracle.matrix(s, metric=metric, p=p, apply_root=False, nthreads=1)
    B = np.empty_like(M)
    for i in range(s.n):
        for j in range(s.n):
            B[i, j] = oracle.integral(*s.pcf(j), *s.pcf(i), metric, p)
    np.testing.assert_array_equal(M, B.T)
    np.testing.assert_array_equal(M, M.T)


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0, 3.5])
def test_triangle_inequality(p):
    s = synth.random_set(30, seed=12, max_len=40)
    D = oracle.matrix(s, metric="lp", p=p)
    lhs = D[:, None, :]
    rhs = D[:, :, None] + D[None, :, :]
    assert np.all(lhs <= rhs * (1 + 1e-12) + 1e-12)


def test_gram_psd_cauchy_schwarz_and_l2_identity():
    s = synth.random_set(40, seed=13, max_len=40)
    G = oracle.matrix(s, metric="gram")
    w = np.linalg.eigvalsh(G)
    assert w.min() >= -1e-10 * w.max()
    d = np.sqrt(np.diag(G))
    assert np.all(np.abs(G) <= np.outer(d, d) * (1 + 1e-12))
    D2 = oracle.matrix(s, metric="l2", apply_root=False)
    recon = np.diag(G)[:, None] + np.diag(G)[None, :] - 2 * G
    scale = np.where(np.outer(d, d) > 0, np.outer(d, d), 1.0)
    assert np.max(np.abs(D2 - recon) / scale) < 1e-12


def test_refinement_invariance_dyadic_bitwise():
    """Sec. 2: a refinement discretizes the same function, so inserting
    breakpoints that keep the value leaves every integral unchanged."""
    s = synth.dyadic(12, seed=5, max_len=20)
    rng = np.random.default_rng(1)
    refined = []
    for i in range(s.n):
        t, v = s.pcf(i)
        extra = np.setdiff1d(rng.integers(1, int(t[-1]) + 10, size=5).astype(float) + 0.5, t)
        tt = np.sort(np.concatenate([t, extra]))
        vv = brute.evaluate(t, v, tt)
        refined.append((tt, vv))
    r = _set_from_pcfs(refined)
    for metric, p in (("l1", 1), ("l2", 2), ("lp", 3), ("gram", 1)):
        a = oracle.matrix(s, metric=metric, p=p, apply_root=False)
        b = oracle.matrix(r, s, metric=metric, p=p, apply_root=False)
        np.testing.assert_array_equal(a, b)


def test_time_scaling_exact():
    s = synth.random_set(20, seed=14, max_len=40)
    scaled = synth.PcfSet(s.offsets, s.times * 8.0, s.values)
    for metric, p in (("l1", 1), ("l2", 2), ("lp", 3.5), ("gram", 1)):
        a = oracle.matrix(s, metric=metric, p=p, apply_root=False)
        b = oracle.matrix(scaled, metric=metric, p=p, apply_root=False)
        np.testing.assert_array_equal(b, a * 8.0)
    a = oracle.matrix(s, metric="lp", p=2.0)
    b = oracle.matrix(scaled, metric="lp", p=2.0)
    np.testing.assert_allclose(b, a * np.sqrt(8.0), rtol=1e-15)


def test_gram_linearity():
    s = synth.random_set(6, seed=15, max_len=30)
    (t0, v0), (t1, v1), (t2, v2) = s.pcf(0), s.pcf(1), s.pcf(2)
    grid = np.union1d(t0, t1)
    vs = brute.evaluate(t0, v0, grid) + 2.5 * brute.evaluate(t1, v1, grid)
    lhs = oracle.integral(grid, vs, t2, v2, "gram")
    rhs = (oracle.integral(t0, v0, t2, v2, "gram")
           + 2.5 * oracle.integral(t1, v1, t2, v2, "gram"))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


# --------------------------------------------------------------------------
# Independent implementations
# --------------------------------------------------------------------------
@pytest.mark.parametrize("metric,p", [("l1", 1), ("l2", 2), ("lp", 3), ("lp", 3.5), ("gram", 1)])
def test_against_union_grid(metric, p):
    s = synth.random_set(25, seed=16, min_len=1, max_len=30)
    a = oracle.matrix(s, metric=metric, p=p)
    b = brute.matrix(s, metric=metric, p=p)
    scale = np.maximum(np.abs(b), 1e-300)
    if metric == "gram":
        d = np.sqrt(np.diag(brute.matrix(s, metric="gram")))
        scale = np.where(np.outer(d, d) > 0, np.outer(d, d), 1.0)
    assert np.max(np.abs(a - b) / scale) < 1e-13


def test_cross_and_row_blocks():
    a = synth.random_set(13, seed=17, max_len=20)
    b = synth.random_set(9, seed=18, max_len=25)
    full = oracle.matrix(a, b, metric="l1")
    np.testing.assert_allclose(full, brute.matrix(a, b, metric="l1"), rtol=1e-13)
    blk = oracle.matrix(a, b, metric="l1", rows=(4, 11))
    np.testing.assert_array_equal(blk, full[4:11])
    pw = oracle.matrix(a, metric="gram")
    np.testing.assert_array_equal(oracle.matrix(a, metric="gram", rows=(3, 7)), pw[3:7])


@pytest.mark.parametrize("metric,p", [("l1", 1), ("l2", 2), ("lp", 3), ("gram", 1)])
def test_exact_rational_tiny(metric, p):
    s = synth.random_set(8, seed=19, min_len=1, max_len=8)
    for i in range(s.n):
        for j in range(s.n):
            ex = brute.exact_integral(*s.pcf(i), *s.pcf(j), metric, p)
            got = oracle.integral(*s.pcf(i), *s.pcf(j), metric, p)
            tol = 1e-14 * max(1.0, abs(float(ex)))
            if metric == "gram":
                na = float(brute.exact_integral(*s.pcf(i), *s.pcf(i), "gram"))
                nb = float(brute.exact_integral(*s.pcf(j), *s.pcf(j), "gram"))
                tol = 1e-14 * max(1.0, np.sqrt(na * nb))
            assert abs(got - float(ex)) <= tol


@pytest.mark.parametrize("metric,p", [("l1", 1), ("l2", 2), ("lp", 3), ("gram", 1)])
def test_dyadic_exact(metric, p):
    """Integer gaps and values: every term and partial sum is an integer, so
    the float64 walk must equal the exact rational integral."""
    s = synth.dyadic(10, seed=21, max_len=12, min_len=1)
    for i in range(s.n):
        for j in range(s.n):
            ex = brute.exact_integral(*s.pcf(i), *s.pcf(j), metric, p)
            assert oracle.integral(*s.pcf(i), *s.pcf(j), metric, p) == float(ex)


def test_tail_rule():
    tf, vf = np.array([0.0, 1.0]), np.array([1.0, 2.0])
    tg, vg = np.array([0.0, 3.0]), np.array([1.0, 2.0])
    assert oracle.integral(tf, vf, tg, vg, "l1") == 2.0      # equal tails: finite
    tg2, vg2 = np.array([0.0, 3.0]), np.array([1.0, 0.0])
    assert oracle.integral(tf, vf, tg2, vg2, "l1") == np.inf
    assert oracle.integral(tf, vf, tg, vg, "gram") == np.inf
    assert oracle.integral(tf, -vf, tg, vg, "gram") == -np.inf
    # a length-1 PCF is a constant function
    assert oracle.integral([0.0], [0.0], [0.0, 2.0], [3.0, 0.0], "l1") == 6.0


def test_merge_steps_is_union_size():
    s = synth.dyadic(10, seed=22, max_len=15)
    for i in range(s.n):
        for j in range(s.n):
            ti, tj = s.pcf(i)[0], s.pcf(j)[0]
            m = oracle.merge_steps(ti, tj)
            assert m == np.union1d(ti, tj).size
            assert m == oracle.rectangles(*s.pcf(i), *s.pcf(j)).shape[0]


# --------------------------------------------------------------------------
# Adjoint
# --------------------------------------------------------------------------
def _loss(s, G, metric, p, apply_root):
    return float(np.sum(G * oracle.matrix(s, metric=metric, p=p, apply_root=apply_root,
                                          nthreads=1)))


@pytest.mark.parametrize("metric,p,root", [("l2", 2, False), ("l1", 1, False),
                                           ("gram", 1, False), ("lp", 3, False),
                                           ("lp", 2.5, True), ("l2", 2, True)])
def test_gradient_central_differences(metric, p, root):
    s = synth.random_set(6, seed=23, min_len=2, max_len=9)
    G = np.random.default_rng(5).standard_normal((s.n, s.n))
    gv, gt = oracle.backward(s, G, metric=metric, p=p, apply_root=root)
    h = 1e-6
    lasts = set((s.offsets[1:] - 1).tolist())
    for k in range(s.nnz):
        if k in lasts:
            continue  # moving a final value makes the integral diverge
        vp, vm = s.values.copy(), s.values.copy()
        vp[k] += h
        vm[k] -= h
        fd = (_loss(synth.PcfSet(s.offsets, s.times, vp), G, metric, p, root)
              - _loss(synth.PcfSet(s.offsets, s.times, vm), G, metric, p, root)) / (2 * h)
        assert fd == pytest.approx(gv[k], rel=1e-5, abs=1e-6), ("value", k)
    starts = set(s.offsets[:-1].tolist())
    for k in range(s.nnz):
        if k in starts:
            assert gt[k] == 0.0
            continue
        tp, tm = s.times.copy(), s.times.copy()
        tp[k] += h
        tm[k] -= h
        fd = (_loss(synth.PcfSet(s.offsets, tp, s.values), G, metric, p, root)
              - _loss(synth.PcfSet(s.offsets, tm, s.values), G, metric, p, root)) / (2 * h)
        assert fd == pytest.approx(gt[k], rel=1e-5, abs=1e-6), ("time", k)


def _exact_loss(pcfs, G, metric):
    n = len(pcfs)
    L = Fraction(0)
    for i in range(n):
        for j in range(n):
            L += G[i][j] * brute.exact_integral(*pcfs[i], *pcfs[j], metric, 2)
    return L


@pytest.mark.parametrize("metric", ["l2", "gram", "l1"])
def test_gradient_dyadic_exact_one_sided(metric):
    """Integer breakpoints with shared times: the value gradient equals the
    exact central difference (the loss is piecewise quadratic in values with
    kinks only at equal values, where |.| has slope 0 in the mean) and the time
    gradient equals the exact left difference quotient."""
    s = synth.dyadic(4, seed=24, max_len=5, min_len=2, max_gap=3, max_abs_value=3)
    rng = np.random.default_rng(6)
    Gi = rng.integers(-8, 9, size=(s.n, s.n))
    G = [[Fraction(int(x), 8) for x in row] for row in Gi]
    gv, gt = oracle.backward(s, Gi / 8.0, metric=metric, p=2.0)
    pcfs = [tuple(map(list, s.pcf(i))) for i in range(s.n)]
    h = Fraction(1, 4)
    base = _exact_loss(pcfs, G, metric)
    for i in range(s.n):
        for k in range(len(pcfs[i][0])):
            t, v = pcfs[i]
            if k < len(t) - 1:  # moving a final value makes the integral diverge
                up = [list(q) for q in pcfs]
                dn = [list(q) for q in pcfs]
                up[i] = (t, v[:k] + [Fraction(v[k]) + h] + v[k + 1:])
                dn[i] = (t, v[:k] + [Fraction(v[k]) - h] + v[k + 1:])
                fd = (_exact_loss(up, G, metric) - _exact_loss(dn, G, metric)) / (2 * h)
                assert float(fd) == gv[s.offsets[i] + k], ("value", i, k)
            if k == 0:
                assert gt[s.offsets[i] + k] == 0.0
                continue
            left = [list(q) for q in pcfs]
            left[i] = (t[:k] + [Fraction(t[k]) - h] + t[k + 1:], v)
            lq = (base - _exact_loss(left, G, metric)) / h
            assert float(lq) == gt[s.offsets[i] + k], ("time", i, k)


# --------------------------------------------------------------------------
# Segment iteration (Alg. 3): single-PCF integrals over [a, b]
# --------------------------------------------------------------------------
def test_segment_integral_closed_forms():
    t, v = _indicator(2.5, 1.0, 4.0)          # 2.5 on [1, 4)
    assert oracle.segment_integral(t, v, "integral") == 7.5
    assert oracle.segment_integral(t, v, "integral", a=2.0, b=3.5) == 2.5 * 1.5
    assert oracle.segment_integral(t, v, "integral", a=0.0, b=0.5) == 0.0
    assert oracle.segment_integral(t, v, "lp", p=3.0, a=0.5, b=10.0) == 2.5 ** 3 * 3.0
    assert oracle.segment_integral([0.0, 1.0], [1.0, 2.0], "integral") == np.inf
    assert oracle.segment_integral([0.0, 1.0], [1.0, 2.0], "integral", b=3.0) == 1.0 + 4.0


@pytest.mark.parametrize("kind,p", [("integral", 1.0), ("lp", 1.0), ("lp", 2.0), ("lp", 3.5)])
def test_segment_integral_against_union_grid(kind, p):
    """The single-PCF integral equals the pair integral against the zero PCF
    (for |f|^p) and the brute-force sum over the clipped breakpoints."""
    s = synth.random_set(40, seed=25, min_len=1, max_len=30)
    rng = np.random.default_rng(2)
    for i in range(s.n):
        t, v = s.pcf(i)
        a = float(rng.uniform(0, t[-1] + 1))
        b = a + float(rng.exponential(5.0))
        grid = np.unique(np.concatenate([t[(t > a) & (t < b)], [a, b]]))
        vals = brute.evaluate(t, v, grid[:-1])
        h = vals if kind == "integral" else np.abs(vals) ** p
        want = float(np.sum(h * np.diff(grid)))
        got = oracle.segment_integral(t, v, kind, p, a, b)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12)
        if kind == "lp":
            full = oracle.segment_integral(t, v, kind, p)
            pair = oracle.integral(t, v, [0.0], [0.0], "lp", p)
            assert full == pytest.approx(pair, rel=1e-13)


# --------------------------------------------------------------------------
# Integration bounds and time-dependent (weighted) integrands
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(12))
def test_bounded_weighted_indicator_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    lo, hi = np.sort(rng.uniform(0, 10, 2))
    lo2, hi2 = np.sort(rng.uniform(0, 10, 2))
    a, b = np.sort(rng.uniform(0, 12, 2))
    lam = [0.0, 0.3, 2.0][seed % 3]
    c, d = rng.normal(size=2) * 2
    tf, vf = _indicator(c, lo, hi)
    tg, vg = _indicator(d, lo2, hi2)

    def wint(x, y):             # int_x^y exp(-lam t) dt
        if y <= x:
            return 0.0
        return (y - x) if lam == 0 else (np.exp(-lam * x) - np.exp(-lam * y)) / lam

    ov = wint(max(lo, lo2, a), min(hi, hi2, b))
    got = oracle.integral_ab(tf, vf, tg, vg, "gram", 1.0, a, b, lam)
    assert got == pytest.approx(c * d * ov, rel=1e-12, abs=1e-12)
    # |f - g|: pieces where only f, only g, or both are on
    f_only = wint(max(lo, a), min(hi, b)) - ov
    g_only = wint(max(lo2, a), min(hi2, b)) - ov
    want = abs(c) * f_only + abs(d) * g_only + abs(c - d) * ov
    assert oracle.integral_ab(tf, vf, tg, vg, "l1", 1.0, a, b, lam) == pytest.approx(
        want, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("lam", [0.25, 1.0, 3.0])
def test_weighted_unbounded_tail_closed_form(lam):
    """f = c on [s, inf), g = d on [0, inf) (neither compact): with the weight
    exp(-lam t) the integrals over [0, inf) are finite and have closed forms."""
    s, c, d = 1.75, 2.5, -0.75
    tf, vf = np.array([0.0, s]), np.array([0.0, c])
    tg, vg = np.array([0.0]), np.array([d])
    es = np.exp(-lam * s)
    got = oracle.integral_ab(tf, vf, tg, vg, "gram", 1.0, 0.0, np.inf, lam)
    assert got == pytest.approx(c * d * es / lam, rel=1e-14)
    got = oracle.integral_ab(tf, vf, tg, vg, "l1", 1.0, 0.0, np.inf, lam)
    assert got == pytest.approx(abs(d) * (1 - es) / lam + abs(c - d) * es / lam, rel=1e-14)
    got = oracle.integral_ab(tf, vf, tg, vg, "l2", 2.0, 0.5, np.inf, lam)
    want = d * d * (np.exp(-lam * 0.5) - es) / lam + (c - d) ** 2 * es / lam
    assert got == pytest.approx(want, rel=1e-14)
    # lam = 0 keeps the unweighted tail rule (reading 2): +inf, and 0 where h = 0
    assert oracle.integral_ab(tf, vf, tg, vg, "l1", 1.0, 0.0, np.inf, 0.0) == np.inf
    assert oracle.integral_ab(tf, vf, tf, vf, "l1", 1.0, 0.0, np.inf, 0.0) == 0.0


def test_bounded_reduces_to_whole_line_and_splits_additively():
    s = synth.random_set(20, seed=26, min_len=1, max_len=30)
    rng = np.random.default_rng(3)
    for i in range(s.n - 1):
        f, g = s.pcf(i), s.pcf(i + 1)
        for m, p in (("l1", 1), ("lp", 3.5), ("gram", 1)):
            assert oracle.integral_ab(*f, *g, m, p) == oracle.integral(*f, *g, m, p)
            c = float(rng.uniform(0.1, 8.0))
            whole = oracle.integral_ab(*f, *g, m, p, 0.0, 20.0, 0.4)
            parts = (oracle.integral_ab(*f, *g, m, p, 0.0, c, 0.4)
                     + oracle.integral_ab(*f, *g, m, p, c, 20.0, 0.4))
            assert parts == pytest.approx(whole, rel=1e-12, abs=1e-12)


def test_weighted_against_quadrature():
    """Independent pin: adaptive quadrature of h(f(t), g(t)) exp(-lam t) over
    each cell of the common refinement."""
    from scipy import integrate
    s = synth.random_set(6, seed=27, min_len=2, max_len=12)
    for i in range(s.n - 1):
        (tf, vf), (tg, vg) = s.pcf(i), s.pcf(i + 1)
        a, b, lam = 0.3, float(max(tf[-1], tg[-1]) + 1.0), 0.7
        grid = np.unique(np.concatenate([tf, tg, [a, b]]))
        grid = grid[(grid >= a) & (grid <= b)]
        want = 0.0
        for x, y in zip(grid[:-1], grid[1:]):
            fv = brute.evaluate(tf, vf, np.array([x]))[0]
            gv = brute.evaluate(tg, vg, np.array([x]))[0]
            want += integrate.quad(lambda t: (fv - gv) ** 2 * np.exp(-lam * t), x, y,
                                   epsabs=1e-14, epsrel=1e-13)[0]
        got = oracle.integral_ab(tf, vf, tg, vg, "l2", 2.0, a, b, lam)
        assert got == pytest.approx(want, rel=1e-10)
        # b = inf: the last cell [t_last, inf) integrated to infinity
        vf2, vg2 = vf.copy(), vg.copy()
        vf2[-1], vg2[-1] = 1.5, -0.5
        grid = np.unique(np.concatenate([tf, tg, [a]]))
        grid = np.append(grid[grid >= a], np.inf)
        want = 0.0
        for x, y in zip(grid[:-1], grid[1:]):
            fv = brute.evaluate(tf, vf2, np.array([x]))[0]
            gv = brute.evaluate(tg, vg2, np.array([x]))[0]
            want += integrate.quad(lambda t: abs(fv - gv) * np.exp(-lam * t), x, y,
                                   epsabs=1e-14, epsrel=1e-13)[0]
        got = oracle.integral_ab(tf, vf2, tg, vg2, "l1", 1.0, a, np.inf, lam)
        assert got == pytest.approx(want, rel=1e-10)
