"""float64 input walked in float32: comparisons exact in float64 (needs a GPU).

The float32 walks of float64 input decide which interval ends first, and
ties (the comparisons of Alg. 1), on order keys ranked from the float64
times, and form each width from the float64 difference of its ends; the
tolerance is the compensated float32 target, 1e-5.  These cases put
many breakpoints of different PCFs inside one float32 ulp, where rounding the
times to float32 would merge and reorder them, and check the result against
the oracle's float64 walk; the rounded form is kept as an explicit opt-in
("*_round" precisions) and is shown to be unable to resolve them.
"""
import numpy as np
import pytest

import oracle
from paper_2404_07183_gb300 import synth

from conftest import gpu_available, max_rel_error

pytestmark = pytest.mark.gpu

TOL = {"f32c": 1e-5, "f32b": 1e-5, "f32": 5e-4}
SCHEDULES = ["tile1024", "tile512x2", "tile512x3", "mergepath", ("tile1024", 8), ("tile512x3", 40)]


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


def subulp_set(n_pcfs=70, seed=201, t0=4096.0):
    """PCFs that are 0 on [0, t_1) with t_1 = t0 + U(0, 1e-3), then hundreds of
    breakpoints spaced 1e-5 * (0.5 + Exp(1)) apart: one float32 ulp at 4096 is
    4.9e-4, so each float32 ulp holds dozens of breakpoints of every PCF.

    The keyed walk carries each time as float32 hi + lo, about 48 bits, so a
    width is exact to about 2^-48 * t (1.5e-11 here); the gaps of a PCF are kept
    above 5e-6 so that the smallest integral (one such gap) stays within the
    1e-5 target.  Widths between breakpoints of different PCFs may be smaller:
    their error is just as small in absolute terms."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(2, 300, n_pcfs)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    t = np.empty(int(offs[-1]))
    v = np.empty(int(offs[-1]))
    for i in range(n_pcfs):
        a, b = int(offs[i]), int(offs[i + 1])
        n = b - a
        t[a] = 0.0
        if n > 1:
            t[a + 1] = t0 + rng.uniform(0.0, 1e-3)
            t[a + 2:b] = t[a + 1] + np.cumsum(1e-5 * (0.5 + rng.exponential(1.0, n - 2)))
        v[a] = 0.0
        v[a + 1:b] = rng.standard_normal(n - 1)
        v[b - 1] = 0.0
    return synth.PcfSet(offs, t, v, "subulp")


@pytest.fixture(scope="module")
def subulp():
    s = subulp_set()
    want = {m: oracle.matrix(s, metric=m) for m in ("l1", "l2", "gram")}
    diag = np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)])
    return s, want, diag


def test_subulp_set_is_what_it_claims(subulp):
    s = subulp[0]
    t32 = s.times.astype(np.float32).astype(np.float64)
    inner = np.ones(s.nnz, bool)
    inner[s.offsets[:-1]] = False
    # most breakpoints share their float32 value with another breakpoint
    _, counts = np.unique(t32[inner], return_counts=True)
    assert np.mean(counts > 1) > 0.9
    assert np.unique(s.times[inner]).size == np.sum(inner)     # distinct in float64


@pytest.mark.parametrize("prec", ["f32c", "f32b", "f32"])
@pytest.mark.parametrize("sched", SCHEDULES, ids=str)
def test_subulp_breakpoints_stay_distinct(pcf, subulp, prec, sched):
    import torch
    s, want, diag = subulp
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise(x, ["l1", "l2", "gram"], precision=prec, out_dtype=torch.float64,
                           schedule=sched)
    for m, g in zip(("l1", "l2", "gram"), got):
        err = max_rel_error(m, g.cpu().numpy(), want[m], diag)
        assert err <= TOL[prec], (m, err)


def test_rounded_times_cannot_resolve_subulp_breakpoints(pcf, subulp):
    """The opt-in rounded form merges the breakpoints: it either reports more
    coincident float32 times than a window holds (reason 7) or is far off."""
    import torch
    s, want, diag = subulp
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    try:
        got = pcf.pcf_pairwise(x, ["l1"], precision="f32c_round", out_dtype=torch.float64)[0]
    except pcf.PcfError as e:
        assert e.detail == 7
        return
    assert max_rel_error("l1", got.cpu().numpy(), want["l1"]) > 1e-3


@pytest.mark.parametrize("prec", ["f32c_round", "f32b_round", "f32_round"])
def test_rounded_times_opt_in_on_ordinary_data(pcf, prec):
    """On data whose breakpoints are far apart in float32 the opt-in rounded
    form still meets its precision's tolerance."""
    import torch
    s = synth.random_set(120, seed=203, min_len=1, max_len=60)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    base = prec.split("_")[0]
    got = pcf.pcf_pairwise(x, ["l1", "gram"], precision=prec, out_dtype=torch.float64)
    diag = np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)])
    for m, g in zip(("l1", "gram"), got):
        err = max_rel_error(m, g.cpu().numpy(), oracle.matrix(s, metric=m), diag)
        assert err <= TOL[base], (m, err)


def test_rounded_times_rejected_with_float64_precision(pcf):
    s = synth.random_set(10, seed=204)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    with pytest.raises(pcf.PcfError):
        pcf.pcf_pairwise(x, ["l1"], precision=pcf.abi.PCF_PREC_F64 | pcf.abi.PCF_PREC_ROUND_TIMES)


@pytest.mark.parametrize("prec", ["f32c", "f32b"])
def test_keyed_dyadic_many_ties_bitwise(pcf, prec):
    """Integer times shared by many PCFs (equal keys across tiles of the key
    sort: about 60,000 interval ends): raw integrals are exact integers, so
    the keyed walk must reproduce the oracle bit for bit."""
    import torch
    s = synth.dyadic(2000, seed=205, max_len=60, min_len=1, max_gap=2, max_abs_value=6)
    assert s.nnz - s.n > 3 * 8192
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise(x, ["l1", ("l2", False), "gram"], precision=prec,
                           out_dtype=torch.float64, schedule="tile512x3")
    for m, g in zip(("l1", ("l2", False), "gram"), got):
        name = m if isinstance(m, str) else m[0]
        root = True if isinstance(m, str) else m[1]
        np.testing.assert_array_equal(g.cpu().numpy(),
                                      oracle.matrix(s, metric=name, apply_root=root))


@pytest.mark.parametrize("sched", ["tile1024", "tile512x3"])
def test_keyed_window_bounds_on_and_between_breakpoints(pcf, sched):
    """Bounds a, b that are breakpoints (integers of a dyadic set) and bounds
    between breakpoints, in the keyed compensated walk: dyadic bounds on
    breakpoints give exact integers, the others meet the tolerance."""
    import torch
    s = synth.dyadic(60, seed=206, max_len=40, min_len=1, final_zero=False)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for (a, b) in ((3.0, 47.0), (2.5, 40.25), (0.0, 19.0), (5.0, np.inf)):
        got = pcf.pcf_pairwise(x, ["l1", ("l2", False), "gram"], precision="f32c",
                               out_dtype=torch.float64, schedule=sched, window=(a, b))
        for (name, root), g in zip((("l1", True), ("l2", False), ("gram", True)), got):
            want = np.array([[oracle.integral_ab(*s.pcf(i), *s.pcf(j), name,
                                                 {"l1": 1.0, "l2": 2.0, "gram": 1.0}[name], a, b)
                              for j in range(s.n)] for i in range(s.n)])
            g = g.cpu().numpy()
            fin = np.isfinite(want)
            np.testing.assert_array_equal(np.isfinite(g), fin)
            np.testing.assert_array_equal(g[fin], want[fin])


def test_keyed_cross_mixed_input_dtypes(pcf):
    """A float32 collection against a float64 one in a float32 walk: both are
    packed with order keys (the float32 times exactly), row blocks reuse B."""
    import torch
    a = synth.random_set(70, seed=207, max_len=60).astype(np.float32)
    b = subulp_set(40, seed=208)
    xa, xb = pcf.PcfTensors.from_numpy(a, "cuda"), pcf.PcfTensors.from_numpy(b, "cuda")
    want = oracle.matrix(a, b, metric="l1")
    out = torch.full((a.n, b.n), np.nan, dtype=torch.float64, device="cuda")
    for r0 in range(0, a.n, 32):
        r1 = min(a.n, r0 + 32)
        pcf.pcf_cross(xa, xb, r0, r1, ["l1"], precision="f32c", out=[out[r0:r1]], ld_out=b.n,
                      reuse_b=r0 > 0)
    assert max_rel_error("l1", out.cpu().numpy(), want) <= 1e-5
