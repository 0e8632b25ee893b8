"""The seeded generators produce valid PCF collections with the stated shapes."""
import numpy as np
import pytest

from paper_2404_07183_gb300 import synth


def _check_valid(s, final_zero=True):
    lens = s.lengths()
    assert np.all(lens >= 1)
    assert s.offsets[0] == 0 and s.offsets[-1] == s.times.size == s.values.size
    starts = s.offsets[:-1]
    assert np.all(s.times[starts] == 0)
    d = np.diff(s.times)
    inner = np.ones(d.size, bool)
    inner[s.offsets[1:-1] - 1] = False
    assert np.all(d[inner] > 0)
    assert np.all(np.isfinite(s.times)) and np.all(np.isfinite(s.values))
    if final_zero:
        assert np.all(s.values[s.offsets[1:] - 1] == 0)


def test_uniform_small_shape_and_determinism():
    a = synth.uniform_small(200)
    b = synth.uniform_small(200)
    _check_valid(a)
    np.testing.assert_array_equal(a.times, b.times)
    assert a.lengths().min() >= 10 and a.lengths().max() <= 100


def test_stable_rank_values():
    s = synth.stable_rank(50)
    _check_valid(s)
    for i in range(s.n):
        t, v = s.pcf(i)
        assert v[0] == 200 and v[-1] == 0
        assert np.all(np.diff(v) <= 0)
        assert np.all(v == np.round(v))
    assert s.lengths().min() >= 50 and s.lengths().max() <= 500


def test_lognormal_lengths_and_float32():
    s = synth.lognormal(3000)
    _check_valid(s)
    assert s.dtype == np.float32
    lens = s.lengths()
    assert lens.min() >= 2 and lens.max() <= 10000
    assert 60 < np.median(lens) < 160


def test_euler_sets():
    a, b = synth.euler(20, n_points=100)
    _check_valid(a)
    _check_valid(b)
    assert a.dtype == np.float32
    assert np.all(a.lengths() == 100)
    assert np.all(np.abs(np.diff(a.values.reshape(20, 100)[:, :-1], axis=1)) <= 3)


def test_appendix_a_and_dyadic():
    _check_valid(synth.appendix_a(30))
    d = synth.dyadic(30, seed=3)
    _check_valid(d)
    assert np.all(d.times == np.round(d.times)) and np.all(np.abs(d.values) <= 16)


def test_gradient_workload():
    s, G = synth.gradient(64)
    _check_valid(s)
    assert G.shape == (64, 64)
