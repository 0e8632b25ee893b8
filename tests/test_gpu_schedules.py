"""Every work decomposition gives the oracle's matrices (needs a GPU).

Schedules: 1024-thread tiles, 512-thread tiles (two CTAs per SM), the
warp-per-pair merge path, and tiles with very small shared-memory windows
(W = 8 and 24) so that every pair crosses many windows.
"""
import numpy as np
import pytest

import oracle
from paper_2404_07183_gb300 import synth

from conftest import gpu_available, max_rel_error

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32c": 1e-5, "f32b": 1e-5, "f32": 5e-4}
SCHEDULES = ["tile1024", "tile512x2", "tile512x3", "mergepath", ("tile1024", 8),
             ("tile512x2", 24), ("tile512x3", 40)]


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


@pytest.fixture(scope="module")
def data():
    rng = np.random.default_rng(11)
    lens = np.concatenate([rng.integers(1, 30, 50), rng.integers(100, 700, 20)])
    s = synth.from_lengths(lens, lambda r, m: r.exponential(1.0, m),
                           lambda r, o: np.where(np.isin(np.arange(o[-1]), o[1:] - 1), 0.0,
                                                 r.standard_normal(o[-1])),
                           rng, np.float64, "mixed")
    want = {m: oracle.matrix(s, metric=m) for m in ("l1", "l2", "gram")}
    diag = np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)])
    return s, want, diag


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32b", "f32"])
@pytest.mark.parametrize("sched", SCHEDULES, ids=str)
def test_schedule_parity(pcf, data, prec, sched):
    import torch
    s, want, diag = data
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise(x, ["l1", "l2", "gram"], precision=prec, out_dtype=torch.float64,
                           schedule=sched)
    for m, g in zip(("l1", "l2", "gram"), got):
        err = max_rel_error(m, g.cpu().numpy(), want[m], diag)
        assert err <= TOL[prec], (m, err)


@pytest.mark.parametrize("sched", SCHEDULES, ids=str)
def test_schedule_dyadic_bitwise(pcf, sched):
    import torch
    s = synth.dyadic(60, seed=81, max_len=120, min_len=1, max_gap=2, max_abs_value=6)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise(x, ["l1", ("l2", False), "gram"], precision="f64",
                           out_dtype=torch.float64, schedule=sched)
    for m, g in zip(["l1", ("l2", False), "gram"], got):
        code = m if isinstance(m, str) else m[0]
        want = oracle.matrix(s, metric=code, apply_root=isinstance(m, str))
        np.testing.assert_array_equal(g.cpu().numpy(), want)


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32c_round"])
@pytest.mark.parametrize("sched", ["tile1024", "tile512x2", ("tile1024", 8), ("tile512x2", 24),
                                   ("tile512x3", 40)], ids=str)
def test_mixed_time_scales_dyadic_bitwise(pcf, prec, sched):
    """Blocks whose PCFs run on time scales 2^-2 .. 2^3 apart (so the rows and
    the columns of a tile fill their windows at different rates and the walks
    that split the window memory between the two sides change the split from
    window to window), with small windows: dyadic data keeps every integral
    exact, so each form must give the oracle's matrices bit for bit."""
    import torch
    s = synth.dyadic(90, seed=83, max_len=150, min_len=1, max_gap=2, max_abs_value=6)
    scale = 2.0 ** np.random.default_rng(84).integers(-2, 4, s.n)
    t = s.times.copy()
    for i in range(s.n):
        t[s.offsets[i]:s.offsets[i + 1]] *= scale[i]
    s = synth.PcfSet(s.offsets, t, s.values)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise(x, ["l1", ("l2", False), "gram"], precision=prec,
                           out_dtype=torch.float64, schedule=sched)
    for m, g in zip(["l1", ("l2", False), "gram"], got):
        code = m if isinstance(m, str) else m[0]
        want = oracle.matrix(s, metric=code, apply_root=isinstance(m, str))
        np.testing.assert_array_equal(g.cpu().numpy(), want)


@pytest.mark.parametrize("sched", ["tile512x2", "mergepath", ("tile1024", 16)], ids=str)
def test_schedule_cross_and_packed(pcf, sched):
    import torch
    a = synth.random_set(50, seed=82, max_len=300)
    b = synth.random_set(37, seed=83, max_len=200)
    xa, xb = pcf.PcfTensors.from_numpy(a, "cuda"), pcf.PcfTensors.from_numpy(b, "cuda")
    got = pcf.pcf_cross(xa, xb, 5, 47, ["l1", ("lp", 3.0)], precision="f64",
                        out_dtype=torch.float64, schedule=sched)
    for m, g in zip(["l1", ("lp", 3.0)], got):
        code, p = (m, 1.0) if isinstance(m, str) else m
        want = oracle.matrix(a, b, metric=code, p=p, rows=(5, 47))
        assert max_rel_error(code, g.cpu().numpy(), want) <= 1e-12
    up = pcf.pcf_pairwise(xa, ["gram"], precision="f32c", layout="upper", schedule=sched,
                          out_dtype=torch.float64)[0].cpu().numpy()
    full = oracle.matrix(a, metric="gram")
    diag = np.diag(full)
    iu = np.triu_indices(a.n)
    scale = np.sqrt(np.outer(diag, diag))[iu]
    assert np.max(np.abs(up - full[iu]) / np.where(scale > 0, scale, 1)) <= 1e-5


def test_bad_schedule_rejected(pcf):
    s = synth.random_set(10, seed=84)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    with pytest.raises(pcf.PcfError):
        pcf.pcf_pairwise(x, ["l1"], schedule=("tile1024", 4))
    with pytest.raises(pcf.PcfError):
        pcf.pcf_pairwise(x, ["l1"], schedule=("tile1024", 1 << 20))


def test_autotune_picks_and_caches(pcf, tmp_path):
    import torch
    from paper_2404_07183_gb300 import autotune
    s = synth.stable_rank(600, seed=85)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    path = str(tmp_path / "tune.json")
    name, timings = autotune.tune_pairwise(x, ["l1", "gram"], "f32c", path=path)
    assert name in {"tile1024", "tile512x2", "tile512x3", "mergepath"} and set(timings) >= {name}
    assert autotune.schedule_for(x, ["gram", "l1"], "f32c", path=path, tune=False) == name
    got = pcf.pcf_pairwise(x, ["l1", "gram"], precision="f32c", out_dtype=torch.float64,
                           schedule=name)
    want = oracle.matrix(s, metric="l1")
    assert max_rel_error("l1", got[0].cpu().numpy(), want) <= 1e-5
