"""Integration bounds [a, b] and exp(-lambda t) weights on the GPU against
the oracle's bounded, time-dependent walk (needs a GPU)."""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_07183_gb300 import synth

from conftest import gpu_available

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32c": 1e-5, "f32b": 1e-5}


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


def _want(a_set, b_set, metric, p, root, lo, hi, lam):
    bb = a_set if b_set is None else b_set
    M = np.empty((a_set.n, bb.n))
    for i in range(a_set.n):
        for j in range(bb.n):
            I = oracle.integral_ab(*a_set.pcf(i), *bb.pcf(j), metric, p, lo, hi, lam)
            M[i, j] = brute.root(metric, p, I) if root and metric != "gram" else I
    return M


def _err(metric, got, want, scale=None):
    if metric == "gram":
        s = np.where(scale > 0, scale, 1.0)
        return float(np.max(np.abs(got - want) / s))
    d = np.abs(got - want)
    s = np.where(want == 0, 1.0, np.abs(want))
    return float(np.max(d / s))


def _gram_scale(a_set, b_set, lo, hi, lam):
    bb = a_set if b_set is None else b_set
    da = np.array([oracle.integral_ab(*a_set.pcf(i), *a_set.pcf(i), "gram", 1, lo, hi, lam)
                   for i in range(a_set.n)])
    db = np.array([oracle.integral_ab(*bb.pcf(j), *bb.pcf(j), "gram", 1, lo, hi, lam)
                   for j in range(bb.n)])
    return np.sqrt(np.outer(np.abs(da), np.abs(db)))


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32b"])
@pytest.mark.parametrize("sched", ["tile1024", "tile512x2", "tile512x3"])
@pytest.mark.parametrize("win", [(1.5, 9.0, 0.0), (0.0, 4.25, 0.0), (2.0, np.inf, 0.0),
                                 (0.5, 30.0, 0.35), (0.0, np.inf, 1.2)], ids=str)
def test_window_pairwise(pcf, prec, sched, win):
    import torch
    if win[2] > 0 and sched != "tile1024":
        pytest.skip("weighted walks run on the 1024-thread tiles")
    # values without a final 0: finite only thanks to b < inf or the weight
    s = synth.random_set(70, seed=111, min_len=1, max_len=60)
    v = s.values.copy()
    v[s.offsets[1:] - 1] = np.random.default_rng(1).normal(size=s.n)
    s = synth.PcfSet(s.offsets, s.times, v)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    metrics = [("l1",), ("l2",), ("gram",), ("lp", 3.5)]
    specs = ["l1", "l2", "gram", ("lp", 3.5)]
    got = pcf.pcf_pairwise(x, specs, precision=prec, out_dtype=torch.float64, schedule=sched,
                           window=win)
    lo, hi, lam = win
    scale = _gram_scale(s, None, lo, hi, lam)
    for m, g in zip(metrics, got):
        name, p = m[0], (m[1] if len(m) > 1 else {"l1": 1, "l2": 2, "gram": 1}[m[0]])
        want = _want(s, None, name, p, True, lo, hi, lam)
        g = g.cpu().numpy()
        if np.isinf(hi) and lam == 0:
            np.testing.assert_array_equal(np.isinf(g), np.isinf(want))
            fin = np.isfinite(want)
            g, want = np.where(fin, g, 0.0), np.where(fin, want, 0.0)
        assert _err(name, g, want, scale) <= TOL[prec], (name, _err(name, g, want, scale))


def test_window_dyadic_bitwise(pcf):
    import torch
    s = synth.dyadic(60, seed=112, max_len=40, min_len=1, final_zero=False)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for sched in ("tile1024", "tile512x3", ("tile512x2", 8)):
        got = pcf.pcf_pairwise(x, ["l1", ("l2", False), "gram"], precision="f64",
                               out_dtype=torch.float64, schedule=sched, window=(3.0, 47.0))
        for (name, root), g in zip((("l1", True), ("l2", False), ("gram", True)), got):
            want = _want(s, None, name, {"l1": 1, "l2": 2, "gram": 1}[name], root, 3.0, 47.0, 0.0)
            np.testing.assert_array_equal(g.cpu().numpy(), want)


def test_window_cross(pcf):
    import torch
    a = synth.random_set(40, seed=113, max_len=50)
    b = synth.random_set(25, seed=114, max_len=80)
    xa, xb = pcf.PcfTensors.from_numpy(a, "cuda"), pcf.PcfTensors.from_numpy(b, "cuda")
    got = pcf.pcf_cross(xa, xb, 3, 37, ["l1", "gram"], precision="f64", out_dtype=torch.float64,
                        window=(0.75, 20.0, 0.1))
    for name, g in zip(("l1", "gram"), got):
        want = _want(a, b, name, 1.0, True, 0.75, 20.0, 0.1)[3:37]
        scale = _gram_scale(a, b, 0.75, 20.0, 0.1)[3:37]
        assert _err(name, g.cpu().numpy(), want, scale) <= 1e-12


def test_window_unsupported_combinations(pcf):
    s = synth.random_set(20, seed=115)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    with pytest.raises(pcf.PcfError) as e:
        pcf.pcf_pairwise(x, ["l1"], schedule="mergepath", window=(1.0, 5.0))
    assert e.value.code == 5
    with pytest.raises(pcf.PcfError) as e:
        pcf.pcf_pairwise(x, ["l1"], schedule="tile512x2", window=(0.0, 5.0, 0.5))
    assert e.value.code == 5
    with pytest.raises(pcf.PcfError):
        pcf.pcf_pairwise(x, ["l1"], window=(5.0, 1.0))
