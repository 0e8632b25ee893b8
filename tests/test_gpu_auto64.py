"""PCF_PREC_AUTO64: the float64 walk for inputs whose dynamic range asks for
it, decided on the device (needs a GPU).

With the bit, a float32 precision runs its float32 walk unless a float64
collection has a time or value outside float32's normal range, or gaps below
2^-30 of their time; then the float64 walk runs instead and its matrices are
those of PCF_PREC_F64 bit for bit.  Ordinary input keeps the float32 walk and
its matrices are those of the plain precision bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2404_07183_gb300 import synth

from conftest import gpu_available, max_rel_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


def _run(pcf, x, prec, metrics=("l1", "l2", "gram"), **kw):
    import torch
    ws = torch.empty(max(pcf.pcf_workspace_size(x, None, prec), 256), dtype=torch.uint8,
                     device="cuda")
    out = pcf.pcf_pairwise(x, list(metrics), precision=prec, out_dtype=torch.float64,
                           workspace=ws, **kw)
    return [o.cpu().numpy() for o in out], pcf.pcf_walk_promoted(ws)


def _huge(seed=301):
    s = synth.random_set(90, seed=seed, min_len=1, max_len=50)
    v = s.values * 1e39                      # beyond FLT_MAX = 3.4e38
    return synth.PcfSet(s.offsets, s.times, v)


def _dense(seed=302):
    """Gaps of 1e-9 at t = 4096: below 2^-30 * 4096 = 3.8e-6."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(2, 40, 60)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    t = np.empty(int(offs[-1]))
    v = rng.standard_normal(int(offs[-1]))
    for i in range(lens.size):
        a, b = int(offs[i]), int(offs[i + 1])
        t[a] = 0.0
        if b - a > 1:
            t[a + 1] = 4096.0 + rng.uniform(0, 1e-6)
            t[a + 2:b] = t[a + 1] + np.cumsum(1e-9 * (1.0 + rng.exponential(1.0, b - a - 2)))
        v[b - 1] = 0.0
    return synth.PcfSet(offs, t, v)


@pytest.mark.parametrize("base", ["f32c", "f32b", "f32"])
@pytest.mark.parametrize("sched", [None, "tile512x3", "mergepath"], ids=str)
def test_ordinary_input_keeps_the_float32_walk(pcf, base, sched):
    s = synth.random_set(110, seed=303, min_len=1, max_len=60)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got, promoted = _run(pcf, x, base + "_auto64", schedule=sched)
    want, _ = _run(pcf, x, base, schedule=sched)
    assert not promoted
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)


@pytest.mark.parametrize("make", [_huge, _dense], ids=["beyond_flt_max", "gaps_below_2^-30"])
@pytest.mark.parametrize("sched", [None, "tile512x2", "mergepath"], ids=str)
def test_dynamic_range_promotes_to_float64(pcf, make, sched):
    s = make()
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got, promoted = _run(pcf, x, "f32c_auto64", schedule=sched)
    want, _ = _run(pcf, x, "f64", schedule=sched)
    assert promoted
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)
    diag = np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)])
    for m, g in zip(("l1", "l2", "gram"), got):
        assert max_rel_error(m, g, oracle.matrix(s, metric=m), diag) <= 1e-12, m


def test_without_the_bit_out_of_range_input_is_rejected(pcf):
    x = pcf.PcfTensors.from_numpy(_huge(), "cuda")
    with pytest.raises(pcf.PcfError) as ei:
        pcf.pcf_pairwise(x, ["l1"], precision="f32c")
    assert ei.value.detail == 6


def test_prepared_workspace_and_windows(pcf):
    """pcf_prepare decides once; PCF_PAIRWISE_PREPARED calls (with a window
    here) walk the form it packed."""
    import torch
    for s, want_promoted in ((synth.random_set(80, seed=304, max_len=40), False), (_dense(), True)):
        x = pcf.PcfTensors.from_numpy(s, "cuda")
        ws = pcf.pcf_prepare(x, "f32c_auto64")
        assert pcf.pcf_walk_promoted(ws) == want_promoted
        ref = pcf.pcf_pairwise(x, ["l1"], precision="f64" if want_promoted else "f32c",
                               out_dtype=torch.float64, window=(0.5, 4096.0000004))[0]
        got = pcf.pcf_pairwise(x, ["l1"], precision="f32c_auto64", out_dtype=torch.float64,
                               workspace=ws, prepared=True, window=(0.5, 4096.0000004))[0]
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_streamed_to_host(pcf):
    import torch
    s = _huge(305)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    host = pcf.pcf_pairwise_to_host(x, ["l1", "gram"], precision="f32c_auto64",
                                    out_dtype=torch.float64, bands=4)
    want = pcf.pcf_pairwise(x, ["l1", "gram"], precision="f64", out_dtype=torch.float64)
    for h, w in zip(host, want):
        np.testing.assert_array_equal(h.numpy(), w.cpu().numpy())


def test_cross_row_blocks_with_a_reused_b(pcf):
    """B is ordinary; the second row block of A holds values beyond float32's
    range, so that block (and only it) promotes, with B packed again."""
    import torch
    a = synth.random_set(64, seed=306, max_len=40)
    v = a.values.copy()
    v[a.offsets[32]:a.offsets[64]] *= 1e39
    a = synth.PcfSet(a.offsets, a.times, v)
    b = synth.random_set(40, seed=307, max_len=50)
    xa, xb = pcf.PcfTensors.from_numpy(a, "cuda"), pcf.PcfTensors.from_numpy(b, "cuda")
    ws = torch.empty(pcf.pcf_workspace_size(xa, xb, "f32c_auto64"), dtype=torch.uint8,
                     device="cuda")
    out = torch.full((a.n, b.n), np.nan, dtype=torch.float64, device="cuda")
    flags = []
    for r0 in (0, 32):
        pcf.pcf_cross(xa, xb, r0, r0 + 32, ["l1"], precision="f32c_auto64", out=[out[r0:r0 + 32]],
                      ld_out=b.n, reuse_b=r0 > 0, workspace=ws)
        flags.append(pcf.pcf_walk_promoted(ws))
    assert flags == [False, True]
    want = oracle.matrix(a, b, metric="l1")
    o = out.cpu().numpy()
    assert max_rel_error("l1", o[:32], want[:32]) <= 1e-5
    assert max_rel_error("l1", o[32:], want[32:]) <= 1e-12
