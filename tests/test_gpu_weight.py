"""Pairwise matrices against a non-negative PCF weight, against the oracle
(needs a GPU).

The GPU moves every breakpoint to W(t) = int_0^t w and walks the moved
collection; the oracle iterates rectangles over the three breakpoint lists
directly.  Tolerances are the per-matrix targets (float64 1e-12, compensated
float32 1e-5).  Weights with zero stretches, compact support (the integrals
stop at W(inf)) and a positive last value (diverging tails stay infinite)
are covered; w = 1 reproduces the unweighted matrices bit for bit, an
indicator weight the windowed ones, and dyadic inputs give exact integers.
"""
import numpy as np
import pytest

import oracle
from paper_2404_07183_gb300 import synth

from conftest import gpu_available, max_rel_error

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32c": 1e-5, "f32b": 1e-5}
METRICS = ["l1", "l2", "gram", ("lp", 3.5)]


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


def _name(m):
    return m if isinstance(m, str) else m[0]


def _p(m):
    return {"l1": 1.0, "l2": 2.0, "gram": 1.0}.get(m, None) if isinstance(m, str) else float(m[1])


def _weight(seed, n=14, t_max=40.0, compact=True):
    rng = np.random.default_rng(seed)
    t = np.concatenate([[0.0], np.sort(rng.uniform(0, t_max, n - 1))])
    v = rng.uniform(0.2, 2.0, n)
    v[rng.random(n) < 0.3] = 0.0
    v[-1] = 0.0 if compact else 0.7
    return t, v


def _scale(s, w):
    return np.array([oracle.integral_w(*s.pcf(i), *s.pcf(i), *w, "gram") for i in range(s.n)])


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32b"])
@pytest.mark.parametrize("compact", [True, False])
def test_weighted_matrices_vs_oracle(pcf, prec, compact):
    import torch
    s = synth.random_set(100, seed=501, min_len=1, max_len=60)
    if not compact:
        v = s.values.copy()                      # unequal tails: some pairs diverge
        v[s.offsets[1:] - 1] = np.random.default_rng(2).integers(-1, 2, s.n)
        s = synth.PcfSet(s.offsets, s.times, v)
    w = _weight(502, compact=compact)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise_weighted(x, w, METRICS, precision=prec, out_dtype=torch.float64)
    diag = _scale(s, w)
    for m, g in zip(METRICS, got):
        want = oracle.matrix_w(s, w, metric=_name(m), p=_p(m))
        g = g.cpu().numpy()
        np.testing.assert_array_equal(np.isinf(g), np.isinf(want))
        fin = np.isfinite(want)
        err = max_rel_error(_name(m), np.where(fin, g, 0.0), np.where(fin, want, 0.0), diag)
        assert err <= TOL[prec], (m, err)


@pytest.mark.parametrize("sched", ["tile1024", "tile512x3", "mergepath", ("tile512x2", 8)], ids=str)
def test_schedules_and_layouts(pcf, sched):
    import torch
    s = synth.random_set(90, seed=503, min_len=1, max_len=50)
    w = _weight(504)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    full = pcf.pcf_pairwise_weighted(x, w, ["l1", "gram"], precision="f32c",
                                     out_dtype=torch.float64, schedule=sched)
    up = pcf.pcf_pairwise_weighted(x, w, ["l1", "gram"], precision="f32c", layout="upper",
                                   out_dtype=torch.float64, schedule=sched)
    iu = np.triu_indices(s.n)
    diag = _scale(s, w)
    for m, f, u in zip(("l1", "gram"), full, up):
        f = f.cpu().numpy()
        np.testing.assert_array_equal(u.cpu().numpy(), f[iu])
        assert max_rel_error(m, f, oracle.matrix_w(s, w, metric=m), diag) <= 1e-5


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_unit_weight_is_the_unweighted_matrix(pcf, prec):
    import torch
    s = synth.random_set(80, seed=505, min_len=1, max_len=40)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise_weighted(x, (np.array([0.0]), np.array([1.0])), METRICS,
                                    precision=prec, out_dtype=torch.float64)
    want = pcf.pcf_pairwise(x, METRICS, precision=prec, out_dtype=torch.float64)
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g.cpu().numpy(), w.cpu().numpy())


def test_indicator_weight_is_the_window(pcf):
    """w = 1 on [a, b), 0 elsewhere: the integrals of [a, b] (dyadic: exact)."""
    import torch
    s = synth.dyadic(60, seed=506, max_len=40, min_len=1, final_zero=False)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for prec in ("f64", "f32c"):
        got = pcf.pcf_pairwise_weighted(x, (np.array([0.0, 3.0, 47.0]), np.array([0.0, 1.0, 0.0])),
                                        ["l1", ("l2", False), "gram"], precision=prec,
                                        out_dtype=torch.float64)
        want = pcf.pcf_pairwise(x, ["l1", ("l2", False), "gram"], precision=prec,
                                out_dtype=torch.float64, window=(3.0, 47.0))
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g.cpu().numpy(), w.cpu().numpy())


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_dyadic_weights_exact(pcf, prec):
    import torch
    s = synth.dyadic(70, seed=507, max_len=40, min_len=1)
    w = (np.array([0.0, 2.0, 5.0, 9.0, 30.0, 41.0]), np.array([1.0, 0.0, 2.0, 3.0, 0.5, 0.0]))
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise_weighted(x, w, ["l1", ("l2", False), "gram"], precision=prec,
                                    out_dtype=torch.float64)
    for (m, root), g in zip((("l1", True), ("l2", False), ("gram", True)), got):
        np.testing.assert_array_equal(g.cpu().numpy(),
                                      oracle.matrix_w(s, w, metric=m, apply_root=root))


def test_float32_input_and_weight(pcf):
    import torch
    s = synth.random_set(70, seed=508, min_len=1, max_len=40).astype(np.float32)
    w = _weight(509)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    wt = pcf.PcfTensors.from_numpy(synth.PcfSet(np.array([0, w[0].size]), w[0], w[1]), "cuda",
                                   dtype=np.float32)
    w32 = (w[0].astype(np.float32), w[1].astype(np.float32))
    got = pcf.pcf_pairwise_weighted(x, wt, ["l1", "gram"], precision="f32c",
                                    out_dtype=torch.float64)
    diag = _scale(s, w32)
    for m, g in zip(("l1", "gram"), got):
        assert max_rel_error(m, g.cpu().numpy(), oracle.matrix_w(s, w32, metric=m), diag) <= 1e-5


@pytest.mark.parametrize("case", ["negative", "t0", "order", "nan"])
def test_invalid_weight_is_reported(pcf, case):
    s = synth.random_set(20, seed=510, max_len=20)
    t, v = np.array([0.0, 1.0, 2.0, 5.0]), np.array([1.0, 2.0, 0.5, 0.0])
    if case == "negative":
        v[2] = -0.5
    elif case == "t0":
        t[0] = 0.5
    elif case == "order":
        t[3] = 2.0
    else:
        v[1] = np.nan
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    with pytest.raises(pcf.PcfError) as ei:
        pcf.pcf_pairwise_weighted(x, (t, v), ["l1"], precision="f64")
    assert ei.value.detail == 10


def test_invalid_collection_reported_before_the_weight_is_applied(pcf):
    s = synth.random_set(20, seed=511, min_len=3, max_len=20)
    t = s.times.copy()
    k = int(s.offsets[4]) + 1
    t[k + 1] = t[k]
    x = pcf.PcfTensors.from_numpy(synth.PcfSet(s.offsets, t, s.values), "cuda")
    with pytest.raises(pcf.PcfError) as ei:
        pcf.pcf_pairwise_weighted(x, _weight(512), ["l1"], precision="f32c")
    assert ei.value.detail == 3 and ei.value.index == k + 1


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_weighted_cross_row_blocks(pcf, prec):
    """Row blocks of a against b, each call moving both to W(t)."""
    import torch
    a = synth.random_set(70, seed=513, min_len=1, max_len=50)
    b = synth.random_set(45, seed=514, min_len=1, max_len=70)
    w = _weight(515)
    xa, xb = pcf.PcfTensors.from_numpy(a, "cuda"), pcf.PcfTensors.from_numpy(b, "cuda")
    out = torch.full((a.n, b.n + 2), np.nan, dtype=torch.float64, device="cuda")
    outs = [out.clone() for _ in range(2)]
    for r0 in range(0, a.n, 32):
        r1 = min(a.n, r0 + 32)
        pcf.pcf_cross_weighted(xa, xb, w, r0, r1, ["l1", "gram"], precision=prec,
                               out=[o[r0:r1] for o in outs], ld_out=b.n + 2)
    da = np.array([oracle.integral_w(*a.pcf(i), *a.pcf(i), *w, "gram") for i in range(a.n)])
    db = np.array([oracle.integral_w(*b.pcf(j), *b.pcf(j), *w, "gram") for j in range(b.n)])
    for m, o in zip(("l1", "gram"), outs):
        o = o.cpu().numpy()
        assert np.all(np.isnan(o[:, b.n:]))
        want = oracle.matrix_w(a, w, b, metric=m)
        if m == "gram":
            scale = np.sqrt(np.outer(da, db))
            err = np.max(np.abs(o[:, :b.n] - want) / np.where(scale > 0, scale, 1.0))
        else:
            err = max_rel_error(m, o[:, :b.n], want)
        assert err <= TOL[prec], (m, err)
    # w = 1: the unweighted cross block bit for bit
    one = (np.array([0.0]), np.array([1.0]))
    got = pcf.pcf_cross_weighted(xa, xb, one, 10, 50, ["l1"], precision=prec,
                                 out_dtype=torch.float64)[0]
    ref = pcf.pcf_cross(xa, xb, 10, 50, ["l1"], precision=prec, out_dtype=torch.float64)[0]
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
