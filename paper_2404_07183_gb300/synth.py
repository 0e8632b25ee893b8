"""Seeded synthetic PCF collections (inputs only; no integral arithmetic here).

Every collection is returned in CSR form: ``offsets`` (int64, N+1 entries,
offsets[0] = 0), ``times`` and ``values`` (nnz entries each).  PCF i owns the
breakpoints ``times[offsets[i]:offsets[i+1]]`` with ``times[offsets[i]] = 0``
and strictly increasing times, and takes ``values[k]`` on
``[times[k], times[k+1])``; the last value holds on ``[t_last, inf)``
(PCF definition and its n x 2 matrix storage, Sec. 2).

The module serves both the CUDA path and the CPU oracle; it draws random
numbers and lays them out, nothing more.  All draws use numpy's PCG64 with a
fixed seed per workload, so the same call always returns the same arrays.

Workloads (sizes and distributions):

* ``uniform_small``  N=1,000, n ~ U{10..100}, gaps Exp(1), values N(0,1),
  final value 0, float64.
* ``stable_rank``    N=20,000, n ~ U{50..500}, gaps Exp(scale 0.1), values
  non-increasing integers from 200 at t=0 down to 0 at the last breakpoint,
  float64 (stable-rank-like curves).
* ``lognormal``      N=100,000, n = clip(round(LogNormal(ln 100, 1)), 2,
  10,000), gaps Exp(1), values N(0,1), final value 0, float32.
* ``gradient``       N=4,096, n ~ U{20..200}, gaps Exp(1), values N(0,1),
  final value 0, float64, plus an N x N weight matrix G ~ N(0,1).
* ``euler``          two sets of 50,000 PCFs, n = 1,000, gaps Exp(1), values
  an integer random walk with steps uniform in {-3,-2,-1,1,2,3}, final value
  set to 0, float32 (Euler-characteristic-curve-like).
* ``appendix_a``     the synthetic recipe of Appendix A: n ~ U{10..1000},
  times |alpha| * (|t~| sorted), alpha, t~, values ~ N(0,1), final value 0.
* ``dyadic``         small integers: gaps in {1..8}, values in [-16, 16],
  so that every integral term is an exact small integer in float64.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "PcfSet", "from_lengths", "uniform_small", "stable_rank", "lognormal",
    "gradient", "euler", "appendix_a", "dyadic", "random_set", "WORKLOADS",
    "subset",
]


class PcfSet:
    """A CSR-packed collection of PCFs (host numpy arrays)."""

    __slots__ = ("offsets", "times", "values", "name")

    def __init__(self, offsets, times, values, name=""):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.times = np.ascontiguousarray(times)
        self.values = np.ascontiguousarray(values)
        self.name = name
        if self.times.dtype != self.values.dtype:
            raise ValueError("times and values must share a dtype")

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    @property
    def dtype(self):
        return self.times.dtype

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def pcf(self, i: int):
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.times[a:b], self.values[a:b]

    def astype(self, dtype) -> "PcfSet":
        t = self.times.astype(dtype)
        v = self.values.astype(dtype)
        if np.dtype(dtype) != self.times.dtype:
            t = _make_strict(self.offsets, t)
        return PcfSet(self.offsets, t, v, self.name)

    def __repr__(self):
        return f"PcfSet({self.name!r}, n={self.n}, nnz={self.nnz}, dtype={self.dtype})"


def subset(s: PcfSet, idx) -> PcfSet:
    """The PCFs ``idx`` of ``s`` (in that order) as a new CSR set."""
    idx = np.asarray(idx, dtype=np.int64)
    lens = s.lengths()[idx]
    offs = np.zeros(idx.size + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    t = np.empty(int(offs[-1]), s.dtype)
    v = np.empty(int(offs[-1]), s.dtype)
    for j, i in enumerate(idx):
        a, b = int(s.offsets[i]), int(s.offsets[i + 1])
        t[offs[j]:offs[j + 1]] = s.times[a:b]
        v[offs[j]:offs[j + 1]] = s.values[a:b]
    return PcfSet(offs, t, v, s.name + "[subset]")


def _offsets(lengths) -> np.ndarray:
    lengths = np.asarray(lengths, dtype=np.int64)
    offs = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=offs[1:])
    return offs


def _segment_cumsum(offsets, gaps):
    """Per-PCF running sums of ``gaps`` with the first entry of each PCF = 0.

    Done PCF by PCF (or as one 2-D cumsum when all lengths agree) so that
    large collections do not lose precision to one long global running sum.
    """
    lens = np.diff(offsets)
    out = np.empty_like(gaps)
    if lens.size and np.all(lens == lens[0]):
        n = int(lens[0])
        g = gaps.reshape(-1, n).copy()
        g[:, 0] = 0.0
        np.cumsum(g, axis=1, out=g)
        out[:] = g.reshape(-1)
        return out
    for i in range(lens.size):
        a, b = int(offsets[i]), int(offsets[i + 1])
        seg = gaps[a:b].copy()
        seg[0] = 0.0
        np.cumsum(seg, out=out[a:b])
    return out


def _make_strict(offsets, t):
    """Nudge times upward by one ulp where rounding made them non-increasing.

    Rounding float64 breakpoints to float32 can merge two close times; the PCF
    contract (strictly increasing, Sec. 2) needs them apart.
    """
    t = t.copy()
    starts = np.zeros(t.size, dtype=bool)
    starts[offsets[:-1][np.diff(offsets) > 0]] = True
    for _ in range(1000):
        bad = np.nonzero((t[1:] <= t[:-1]) & ~starts[1:])[0] + 1
        if bad.size == 0:
            return t
        t[bad] = np.nextafter(t[bad - 1], np.array(np.inf, dtype=t.dtype))
    raise RuntimeError("could not make times strictly increasing")


def from_lengths(lengths, gap_sampler, value_sampler, rng, dtype=np.float64,
                 name="") -> PcfSet:
    offs = _offsets(lengths)
    nnz = int(offs[-1])
    gaps = gap_sampler(rng, nnz)
    times = _segment_cumsum(offs, gaps.astype(np.float64))
    values = value_sampler(rng, offs).astype(np.float64)
    if np.dtype(dtype) != np.float64:
        times = _make_strict(offs, times.astype(dtype))
        values = values.astype(dtype)
    else:
        times = _make_strict(offs, times)
    return PcfSet(offs, times, values, name)


def _normal_last_zero(rng, offs):
    v = rng.standard_normal(int(offs[-1]))
    v[offs[1:] - 1] = 0.0
    return v


def uniform_small(n_pcfs=1000, seed=1001, dtype=np.float64) -> PcfSet:
    """N PCFs with n ~ U{10..100}, Exp(1) gaps, N(0,1) values, last value 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(10, 100, size=n_pcfs, endpoint=True)
    return from_lengths(lens, lambda r, m: r.exponential(1.0, m),
                        _normal_last_zero, rng, dtype, "uniform_small")


def stable_rank(n_pcfs=20000, seed=1002, dtype=np.float64) -> PcfSet:
    """Stable-rank-like curves: n ~ U{50..500}, Exp(scale 0.1) gaps,
    non-increasing integer values from 200 at t=0 to 0 at the last point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(50, 500, size=n_pcfs, endpoint=True)

    def values(r, offs):
        v = np.empty(int(offs[-1]))
        for i in range(offs.size - 1):
            a, b = int(offs[i]), int(offs[i + 1])
            mid = np.sort(r.integers(0, 200, size=b - a - 2, endpoint=True))[::-1]
            v[a] = 200.0
            v[a + 1:b - 1] = mid
            v[b - 1] = 0.0
        return v

    return from_lengths(lens, lambda r, m: r.exponential(0.1, m), values, rng,
                        dtype, "stable_rank")


def lognormal(n_pcfs=100000, seed=1003, dtype=np.float32, max_len=10000) -> PcfSet:
    """Uneven lengths: n = clip(round(LogNormal(ln 100, 1)), 2, 10000)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = np.clip(np.rint(rng.lognormal(np.log(100.0), 1.0, size=n_pcfs)), 2,
                   max_len).astype(np.int64)
    return from_lengths(lens, lambda r, m: r.exponential(1.0, m),
                        _normal_last_zero, rng, dtype, "lognormal")


def gradient(n_pcfs=4096, seed=1004, dtype=np.float64):
    """PCFs for the adjoint workload plus the weight matrix G ~ N(0,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(20, 200, size=n_pcfs, endpoint=True)
    s = from_lengths(lens, lambda r, m: r.exponential(1.0, m),
                     _normal_last_zero, rng, dtype, "gradient")
    g = np.random.Generator(np.random.PCG64(seed + 1)).standard_normal(
        (n_pcfs, n_pcfs))
    return s, g


def euler(n_pcfs=50000, seed=1005, dtype=np.float32, n_points=1000):
    """Two sets (A, B) of Euler-curve-like PCFs: integer random walks with
    steps uniform in {-3..-1, 1..3} at Exp(1) times, last value 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    steps = np.array([-3, -2, -1, 1, 2, 3], dtype=np.float64)
    for tag in ("A", "B"):
        lens = np.full(n_pcfs, n_points, dtype=np.int64)

        def values(r, offs, n=n_points):
            jumps = steps[r.integers(0, 6, size=(offs.size - 1, n))]
            jumps[:, 0] = 0.0
            v = np.cumsum(jumps, axis=1)
            v[:, -1] = 0.0
            return v.reshape(-1)

        out.append(from_lengths(lens, lambda r, m: r.exponential(1.0, m), values,
                                rng, dtype, "euler_" + tag))
    return out[0], out[1]


def appendix_a(n_pcfs=50000, seed=1006, dtype=np.float64) -> PcfSet:
    """Appendix A recipe: n ~ U{10..1000}; times |alpha| * sorted |t~|
    (alpha, t~ ~ N(0,1)); values N(0,1) with the final value 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(10, 1000, size=n_pcfs, endpoint=True)
    offs = _offsets(lens)
    nnz = int(offs[-1])
    t = np.empty(nnz)
    for i in range(n_pcfs):
        a, b = int(offs[i]), int(offs[i + 1])
        alpha = abs(rng.standard_normal())
        tt = np.sort(np.abs(rng.standard_normal(b - a - 1)))
        t[a] = 0.0
        t[a + 1:b] = alpha * tt
    v = _normal_last_zero(rng, offs)
    t = _make_strict(offs, t.astype(dtype))
    return PcfSet(offs, t, v.astype(dtype), "appendix_a")


def dyadic(n_pcfs=64, seed=7, max_len=64, min_len=1, dtype=np.float64,
           max_gap=8, max_abs_value=16, final_zero=True) -> PcfSet:
    """Small-integer PCFs: gaps in {1..max_gap}, values in
    [-max_abs_value, max_abs_value].  Every partial sum of every integral of
    such PCFs (p = 1, 2, 3 and the inner product) is an integer far below
    2**53, so float64 arithmetic on them is exact in any order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(min_len, max_len, size=n_pcfs, endpoint=True)
    offs = _offsets(lens)
    nnz = int(offs[-1])
    gaps = rng.integers(1, max_gap, size=nnz, endpoint=True).astype(np.float64)
    t = _segment_cumsum(offs, gaps)
    v = rng.integers(-max_abs_value, max_abs_value, size=nnz,
                     endpoint=True).astype(np.float64)
    if final_zero:
        v[offs[1:] - 1] = 0.0
    return PcfSet(offs, t.astype(dtype), v.astype(dtype), "dyadic")


def random_set(n_pcfs, seed, min_len=1, max_len=40, dtype=np.float64,
               gap_scale=1.0) -> PcfSet:
    """Generic small random set (Exp gaps, N(0,1) values, last value 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(min_len, max_len, size=n_pcfs, endpoint=True)
    return from_lengths(lens, lambda r, m: r.exponential(gap_scale, m),
                        _normal_last_zero, rng, dtype, "random")


WORKLOADS = {
    "uniform_small": uniform_small,
    "stable_rank": stable_rank,
    "lognormal": lognormal,
    "gradient": gradient,
    "euler": euler,
    "appendix_a": appendix_a,
}
