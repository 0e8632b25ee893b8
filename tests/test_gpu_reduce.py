"""Reductions (Sec. 4: ReducePair of Alg. 4, binary reduction trees; mean and
standard deviation of Sec. 2.1) and combinations on the GPU against the
oracle (needs a GPU).  Both sides reduce in float64 with the same tree, so
offsets, times and values must agree bit for bit."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2404_07183_gb300 import synth

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


def _host(res):
    return (res.offsets.cpu().numpy(), res.times.cpu().numpy(), res.values.cpu().numpy())


def _assert_same(got, want):
    for g, w, what in zip(got, want, ("offsets", "times", "values")):
        np.testing.assert_array_equal(g, w, err_msg=what)


def _with_repeats(s, seed):
    """Some consecutive values repeated (non-canonical input rows)."""
    v = s.values.copy()
    rng = np.random.default_rng(seed)
    for i in range(s.n):
        a, b = int(s.offsets[i]), int(s.offsets[i + 1])
        for k in range(a + 1, b):
            if rng.random() < 0.15:
                v[k] = v[k - 1]
    return synth.PcfSet(s.offsets, s.times, v)


@pytest.mark.parametrize("red", ["sum", "mean", "max", "min", "std"])
@pytest.mark.parametrize("m,groups,max_len", [(1, 5, 30), (2, 7, 40), (3, 4, 25), (5, 6, 60),
                                              (8, 3, 17), (13, 2, 80), (64, 2, 50)])
def test_reduce_bitwise(pcf, red, m, groups, max_len):
    if red == "std" and m < 2:
        pytest.skip("the sample standard deviation needs m >= 2")
    s = _with_repeats(synth.random_set(m * groups, seed=200 + m, min_len=1, max_len=max_len),
                      seed=m)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = _host(pcf.pcf_reduce(x, m, red))
    _assert_same(got, oracle.reduce(s, m, red))


@pytest.mark.parametrize("red", ["mean", "std", "max"])
def test_reduce_float32_input(pcf, red):
    s = synth.random_set(40, seed=211, min_len=1, max_len=50).astype(np.float32)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = _host(pcf.pcf_reduce(x, 10, red))
    _assert_same(got, oracle.reduce(s, 10, red))       # float32 rows widen exactly


def test_reduce_shared_breakpoints_dyadic(pcf):
    """Integer breakpoints shared by many members and sums that cancel: the
    drop rule of Alg. 4 decides most rows."""
    s = synth.dyadic(48, seed=212, max_len=30, max_gap=2, max_abs_value=2, final_zero=False)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for red in ("sum", "mean", "std", "max", "min"):
        _assert_same(_host(pcf.pcf_reduce(x, 6, red)), oracle.reduce(s, 6, red))
        _assert_same(_host(pcf.pcf_reduce(x, 48, red)), oracle.reduce(s, 48, red))


@pytest.mark.parametrize("red", ["mean", "std"])
def test_reduce_many_chunks_and_long_pcfs(pcf, red):
    """PCFs of thousands of breakpoints: single merges span several CTAs'
    chunks of merge positions, and tree levels span many chunks."""
    a = synth.random_set(24, seed=213, min_len=2000, max_len=6000)
    b = synth.random_set(40, seed=214, min_len=1, max_len=300)
    s = synth.subset(synth.PcfSet(np.concatenate([a.offsets, a.offsets[-1] + b.offsets[1:]]),
                                  np.concatenate([a.times, b.times]),
                                  np.concatenate([a.values, b.values])), np.arange(64))
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for m in (64, 16, 3 if red == "std" else 1):
        if 64 % m:
            continue
        _assert_same(_host(pcf.pcf_reduce(x, m, red)), oracle.reduce(s, m, red))


def test_reduce_stable_rank_groups(pcf):
    """The stable-rank recipe (integer step values that often coincide)."""
    s = synth.stable_rank(600, seed=215)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for red, m in (("mean", 100), ("std", 30), ("max", 600)):
        _assert_same(_host(pcf.pcf_reduce(x, m, red)), oracle.reduce(s, m, red))


@pytest.mark.parametrize("op", ["add", "sub", "mul", "max", "min", "sqdiff"])
def test_combine_pairs_and_broadcast(pcf, op):
    a = _with_repeats(synth.random_set(37, seed=216, min_len=1, max_len=70), 5)
    b = synth.random_set(37, seed=217, min_len=1, max_len=45)
    xa, xb = pcf.PcfTensors.from_numpy(a, "cuda"), pcf.PcfTensors.from_numpy(b, "cuda")
    got = _host(pcf.pcf_combine(xa, xb, op))
    offs, ts, vs = [0], [], []
    for i in range(a.n):
        t, v = oracle.reduce_pair(*a.pcf(i), *b.pcf(i), op)
        ts.append(t); vs.append(v); offs.append(offs[-1] + t.size)
    _assert_same(got, (np.array(offs), np.concatenate(ts), np.concatenate(vs)))
    one = synth.subset(b, [3])
    got = _host(pcf.pcf_combine(xa, pcf.PcfTensors.from_numpy(one, "cuda"), op))
    offs, ts, vs = [0], [], []
    for i in range(a.n):
        t, v = oracle.reduce_pair(*a.pcf(i), *one.pcf(0), op)
        ts.append(t); vs.append(v); offs.append(offs[-1] + t.size)
    _assert_same(got, (np.array(offs), np.concatenate(ts), np.concatenate(vs)))


def test_combine_cancellation_gives_one_row(pcf):
    a = synth.random_set(20, seed=218, min_len=1, max_len=30)
    x = pcf.PcfTensors.from_numpy(a, "cuda")
    off, t, v = _host(pcf.pcf_combine(x, x, "sub"))
    np.testing.assert_array_equal(off, np.arange(21))
    np.testing.assert_array_equal(t, np.zeros(20))
    np.testing.assert_array_equal(v, np.zeros(20))


def test_reduce_errors(pcf):
    import torch
    from paper_2404_07183_gb300 import abi, api
    s = synth.random_set(12, seed=219, min_len=2, max_len=30)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    with pytest.raises(ValueError):
        pcf.pcf_reduce(x, 5, "mean")
    with pytest.raises(pcf.PcfError):
        pcf.pcf_reduce(x, 1, "std")
    # invalid rows are reported like pcf_pairwise's
    t = s.times.copy()
    t[5] = t[4]
    bad = pcf.PcfTensors.from_numpy(synth.PcfSet(s.offsets, t, s.values), "cuda")
    with pytest.raises(pcf.PcfError) as e:
        pcf.pcf_reduce(bad, 4, "sum")
    assert e.value.code == abi.PCF_EINVAL and e.value.detail == 3 and e.value.index == 5
    # a workspace sized for fewer intermediate rows than the std needs
    ws = torch.empty(api.pcf_reduce_workspace_size(x, 12, "std", std_rows=x.nnz),
                     dtype=torch.uint8, device="cuda")
    with pytest.raises(pcf.PcfError) as e:
        pcf.pcf_reduce(x, 12, "std", workspace=ws)
    assert e.value.code == abi.PCF_ENOWS and e.value.detail == 8
    # an output with too little capacity
    lib = abi.load()
    ws = torch.empty(api.pcf_reduce_workspace_size(x, 12, "sum"), dtype=torch.uint8,
                     device="cuda")
    out, off, tt, vv = api._csr_out(1, 3, "cuda")
    cx = x.csr()
    rc = lib.pcf_reduce(ctypes.byref(cx), 12, abi.PCF_RED_SUM, ctypes.byref(out),
                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), api._stream_handle(None))
    assert rc == abi.PCF_OK
    with pytest.raises(pcf.PcfError) as e:
        api.pcf_check(ws)
    assert e.value.code == abi.PCF_ENOWS and e.value.detail == 8
    # the same workspace works again afterwards
    got = _host(pcf.pcf_reduce(x, 12, "sum", workspace=ws))
    _assert_same(got, oracle.reduce(s, 12, "sum"))


def test_reduce_counters(pcf):
    import torch
    from paper_2404_07183_gb300 import api
    s = synth.random_set(16, seed=220, min_len=1, max_len=40)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    ws = torch.empty(api.pcf_reduce_workspace_size(x, 2, "sum"), dtype=torch.uint8, device="cuda")
    res = pcf.pcf_reduce(x, 2, "sum", workspace=ws)
    assert api.pcf_reduce_counters(ws) == (s.nnz, res.nnz)       # one level: every row once
    res = pcf.pcf_reduce(x, 16, "sum", workspace=ws)
    pos, rows = api.pcf_reduce_counters(ws)
    assert pos >= s.nnz and rows >= res.nnz and pos - s.nnz == rows - res.nnz
    a, b = synth.subset(s, range(8)), synth.subset(s, range(8, 16))
    xa, xb = pcf.PcfTensors.from_numpy(a, "cuda"), pcf.PcfTensors.from_numpy(b, "cuda")
    nbytes = 1 << 20
    wsc = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    res = pcf.pcf_combine(xa, xb, "max", workspace=wsc)
    assert api.pcf_reduce_counters(wsc) == (a.nnz + b.nnz, res.nnz)


def test_negative_zero_t0(pcf):
    s = synth.PcfSet([0, 2, 4, 5], np.array([-0.0, 1.0, 0.0, 2.0, -0.0]),
                     np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for red, m in (("sum", 1), ("mean", 1), ("sum", 3), ("std", 3), ("min", 3)):
        got = _host(pcf.pcf_reduce(x, m, red))
        _assert_same(got, oracle.reduce(s, m, red))
        assert not np.any(np.signbit(got[1]))


def test_bounded_wait_gives_up(pcf):
    """The look-back wait of the reductions is bounded: with a predecessor
    that never publishes, it records reason 9 and pcf_check reports
    PCF_ETIMEOUT; the context stays usable."""
    import time

    import torch
    from paper_2404_07183_gb300 import abi, api
    lib = abi.load()
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    rc = lib.pcf_selftest_wait_timeout(1000, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       api._stream_handle(None))
    assert rc == abi.PCF_OK
    with pytest.raises(pcf.PcfError) as e:
        api.pcf_check(ws)
    assert e.value.code == abi.PCF_ETIMEOUT and e.value.detail == 9
    assert time.perf_counter() - t0 < 10.0
    # the device is still fine afterwards
    s = synth.random_set(8, seed=221, max_len=20)
    got = _host(pcf.pcf_reduce(pcf.PcfTensors.from_numpy(s, "cuda"), 4, "mean"))
    _assert_same(got, oracle.reduce(s, 4, "mean"))


def test_reduce_benchmark_size_sampled(pcf):
    """The benchmarked reduction input (stable-rank N = 20,480): every group is
    reduced on the GPU, a sample of groups by the oracle; identical bits."""
    s = synth.stable_rank(n_pcfs=20480)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for red, m, groups in (("mean", 128, (0, 77, 159)), ("std", 16, (0, 555, 1279))):
        r = pcf.pcf_reduce(x, m, red)
        off, t, v = (r.offsets.cpu().numpy(), r.times.cpu().numpy(), r.values.cpu().numpy())
        for g in groups:
            sub = synth.subset(s, np.arange(g * m, (g + 1) * m))
            wo, wt, wv = oracle.reduce(sub, m, red)
            np.testing.assert_array_equal(t[off[g]:off[g + 1]], wt)
            np.testing.assert_array_equal(v[off[g]:off[g + 1]], wv)
