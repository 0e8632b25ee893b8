"""Pins of the oracle's reductions (Sec. 4: ReducePair of Alg. 4 and binary
reduction trees; mean and sample standard deviation of Sec. 2.1) against
brute-force evaluation on the common refinement, exact dyadic arithmetic,
and hand-built cases (CPU only)."""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_07183_gb300 import synth


def _groups(s, m):
    for g in range(s.n // m):
        yield [s.pcf(g * m + i) for i in range(m)]


def _pcfs(out):
    off, t, v = out
    return [(t[off[g]:off[g + 1]], v[off[g]:off[g + 1]]) for g in range(off.size - 1)]


def _grid(members):
    return np.unique(np.concatenate([np.asarray(t, np.float64) for t, _ in members]))


def _values_on(members, grid):
    return np.stack([brute.evaluate(t, v, grid) for t, v in members])


def _check_canonical(t, v, members):
    assert t[0] == 0.0
    assert np.all(np.diff(t) > 0)
    assert np.all(v[1:] != v[:-1])                 # repeated values dropped (Alg. 4)
    assert np.all(np.isin(t, _grid(members)))      # breakpoints from the inputs only


def _probe(grid):
    """The breakpoints and the midpoints between them (and one point past the end)."""
    mids = 0.5 * (grid[1:] + grid[:-1])
    return np.concatenate([grid, mids, [grid[-1] + 1.0]])


# ----------------------------------------------------------------- ReducePair
def test_reduce_pair_hand_example():
    # f = 1 on [0,1), 2 on [1,2), 0 after; g = 3 on [0,1.5), 1 after
    t, v = oracle.reduce_pair([0, 1, 2], [1, 2, 0], [0, 1.5], [3, 1], "add")
    np.testing.assert_array_equal(t, [0, 1, 1.5, 2])
    np.testing.assert_array_equal(v, [4, 5, 3, 1])


def test_reduce_pair_drops_repeated_values_and_keeps_t0():
    # f + g is 3 everywhere although both change at t = 1
    t, v = oracle.reduce_pair([0, 1], [1, 2], [0, 1], [2, 1], "add")
    np.testing.assert_array_equal(t, [0])
    np.testing.assert_array_equal(v, [3])
    # a zero value at t = 0 is still inserted (the t = 0 rule of Alg. 4)
    t, v = oracle.reduce_pair([0, 2], [0, 1], [0, 3], [0, 0], "max")
    np.testing.assert_array_equal(t, [0, 2])
    np.testing.assert_array_equal(v, [0, 1])
    # the comparison is with the previous rectangle, not the last inserted row
    t, v = oracle.reduce_pair([0, 1, 2, 3], [5, 5, 7, 5], [0], [0], "add")
    np.testing.assert_array_equal(t, [0, 2, 3])
    np.testing.assert_array_equal(v, [5, 7, 5])


@pytest.mark.parametrize("op,fn", [("add", np.add), ("sub", np.subtract), ("mul", np.multiply),
                                   ("max", np.maximum), ("min", np.minimum),
                                   ("sqdiff", lambda a, b: (a - b) * (a - b))])
def test_reduce_pair_pointwise(op, fn):
    s = synth.random_set(40, seed=31, min_len=1, max_len=30)
    for i in range(0, s.n - 1, 2):
        f, g = s.pcf(i), s.pcf(i + 1)
        t, v = oracle.reduce_pair(*f, *g, op)
        grid = brute.union_grid(f[0], g[0])
        x = _probe(grid)
        want = fn(brute.evaluate(*f, x), brute.evaluate(*g, x))
        np.testing.assert_array_equal(brute.evaluate(t, v, x), want)   # one operation: exact
        _check_canonical(t, v, [f, g])
        assert t.size <= f[0].size + g[0].size


def test_reduce_pair_union_size_when_values_differ():
    """Distinct breakpoints and values that never repeat: every point of the
    union survives (|T_f u T_g| rows)."""
    f = (np.array([0.0, 1.0, 3.0]), np.array([1.0, 2.0, 4.0]))
    g = (np.array([0.0, 2.0]), np.array([10.0, 20.0]))
    t, v = oracle.reduce_pair(*f, *g, "add")
    np.testing.assert_array_equal(t, [0, 1, 2, 3])
    np.testing.assert_array_equal(v, [11, 12, 22, 24])


# ----------------------------------------------------------------- trees
@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 13])
def test_mean_pointwise(m):
    s = synth.random_set(4 * m, seed=32 + m, min_len=1, max_len=25)
    out = _pcfs(oracle.reduce(s, m, "mean"))
    for (t, v), members in zip(out, _groups(s, m)):
        x = _probe(_grid(members))
        vals = _values_on(members, x)
        want = vals.sum(axis=0) / m
        got = brute.evaluate(t, v, x)
        scale = np.abs(vals).sum(axis=0) / m
        assert np.all(np.abs(got - want) <= 4e-16 * np.log2(2 * m) * scale + 1e-300)
        if m > 1 or np.all(members[0][1][1:] != members[0][1][:-1]):
            _check_canonical(t, v, members)


def test_sum_dyadic_exact_and_order_free():
    """Small integers: every partial sum is exact, so the tree, a sequential
    fold and numpy give the same PCF bit for bit."""
    s = synth.dyadic(8 * 6, seed=33, max_len=30, final_zero=False)
    out = _pcfs(oracle.reduce(s, 8, "sum"))
    mean = _pcfs(oracle.reduce(s, 8, "mean"))
    for (t, v), (tm, vm), members in zip(out, mean, _groups(s, 8)):
        x = _probe(_grid(members))
        vals = _values_on(members, x)
        np.testing.assert_array_equal(brute.evaluate(t, v, x), vals.sum(axis=0))
        np.testing.assert_array_equal(brute.evaluate(tm, vm, x), vals.sum(axis=0) / 8)
        # sequential fold with ReducePair (the O(nM) order of Sec. 4)
        acc = members[0]
        for f in members[1:]:
            acc = oracle.reduce_pair(*acc, *f, "add")
        np.testing.assert_array_equal(acc[0], t)
        np.testing.assert_array_equal(acc[1], v)


def test_tree_shape_pairs_neighbours():
    """The tree pairs (0,1), (2,3), ... level by level with an odd last item
    moving up: for m = 3 the sum is (f0 + f1) + f2, which differs in the last
    bit from f0 + (f1 + f2) on these values."""
    s = synth.PcfSet([0, 1, 2, 3], np.zeros(3), np.array([1.0, 2.0 ** -53, 2.0 ** -53]))
    off, t, v = oracle.reduce(s, 3, "sum")
    assert v[0] == (1.0 + 2.0 ** -53) + 2.0 ** -53 == 1.0
    assert 1.0 + (2.0 ** -53 + 2.0 ** -53) != 1.0                 # the other order


@pytest.mark.parametrize("red,fn", [("max", np.max), ("min", np.min)])
def test_max_min_exact(red, fn):
    s = synth.random_set(5 * 7, seed=34, min_len=1, max_len=20)
    for (t, v), members in zip(_pcfs(oracle.reduce(s, 7, red)), _groups(s, 7)):
        x = _probe(_grid(members))
        np.testing.assert_array_equal(brute.evaluate(t, v, x), fn(_values_on(members, x), axis=0))
        _check_canonical(t, v, members)


@pytest.mark.parametrize("m", [2, 3, 6, 11])
def test_std_against_numpy(m):
    s = synth.random_set(3 * m, seed=35 + m, min_len=1, max_len=20)
    for (t, v), members in zip(_pcfs(oracle.reduce(s, m, "std")), _groups(s, m)):
        x = _probe(_grid(members))
        vals = _values_on(members, x)
        want = vals.std(axis=0, ddof=1)              # unbiased: 1 / (m - 1)
        got = brute.evaluate(t, v, x)
        scale = np.sqrt((vals ** 2).sum(axis=0) / (m - 1))
        assert np.all(np.abs(got - want) <= 1e-13 * scale + 1e-300)
        assert t[0] == 0 and np.all(np.diff(t) > 0) and np.all(v[1:] != v[:-1])
        assert np.all(np.isin(t, _grid(members)))


def test_std_special_cases():
    # four identical members (the mean is then exact): std 0 everywhere, one row
    one = synth.random_set(1, seed=36, min_len=5, max_len=5)
    t0, v0 = one.pcf(0)
    s = synth.PcfSet([0, 5, 10, 15, 20], np.tile(t0, 4), np.tile(v0, 4))
    off, t, v = oracle.reduce(s, 4, "std")
    np.testing.assert_array_equal(t, [0.0])
    np.testing.assert_array_equal(v, [0.0])
    # two constants a, b: std = |a - b| / sqrt(2)
    s = synth.PcfSet([0, 1, 2], np.zeros(2), np.array([3.0, -1.0]))
    off, t, v = oracle.reduce(s, 2, "std")
    assert v[0] == pytest.approx(4.0 / np.sqrt(2.0), rel=1e-15)
    # indicators of [0,1) and [0,2): mean 1, 0.5, 0; std 0, 1/sqrt(2), 0
    s = synth.PcfSet([0, 2, 4], np.array([0.0, 1.0, 0.0, 2.0]), np.array([1.0, 0.0, 1.0, 0.0]))
    off, t, v = oracle.reduce(s, 2, "std")
    np.testing.assert_array_equal(t, [0.0, 1.0, 2.0])
    np.testing.assert_allclose(v, [0.0, np.sqrt(0.5), 0.0], rtol=1e-15)


def test_group_size_one():
    s = synth.random_set(6, seed=37, min_len=1, max_len=9)
    off, t, v = oracle.reduce(s, 1, "sum")
    np.testing.assert_array_equal(off, s.offsets)
    np.testing.assert_array_equal(t, s.times)
    np.testing.assert_array_equal(v, s.values)
    with pytest.raises(ValueError):
        oracle.reduce(s, 4, "mean")


def test_negative_zero_t0_reads_as_zero():
    """t_0 = -0.0 is accepted as 0; every result carries +0.0 there."""
    s = synth.PcfSet([0, 2, 4], np.array([-0.0, 1.0, 0.0, 2.0]), np.array([1.0, 2.0, 3.0, 4.0]))
    for red, m in (("sum", 1), ("mean", 1), ("sum", 2), ("std", 2), ("max", 2)):
        off, t, v = oracle.reduce(s, m, red)
        assert np.all(np.signbit(t) == False), (red, m, t)    # noqa: E712
