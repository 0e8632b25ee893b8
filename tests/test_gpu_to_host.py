"""Pairwise matrices streamed to page-locked host memory band by band
(needs a GPU): the host copies equal the device matrices of pcf_pairwise bit
for bit, for every band count and schedule, and match the oracle."""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_07183_gb300 import synth

from conftest import gpu_available, max_rel_error

pytestmark = pytest.mark.gpu

METRICS = ["l1", "l2", "gram"]


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


@pytest.fixture(scope="module")
def stable700(pcf):
    s = synth.stable_rank(n_pcfs=700, seed=71)      # 22 blocks of 32, the last ragged
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    return s, x


@pytest.mark.parametrize("schedule", [None, "tile512x3", "tile512x2", "tile1024"])
@pytest.mark.parametrize("bands", [0, 1, 3, 7, 1000])
def test_to_host_equals_device_matrices(pcf, stable700, schedule, bands):
    import torch
    s, x = stable700
    want = pcf.pcf_pairwise(x, METRICS, precision="f32c", schedule=schedule)
    got = pcf.pcf_pairwise_to_host(x, METRICS, precision="f32c", bands=bands, schedule=schedule)
    for w, g in zip(want, got):
        assert g.is_pinned() and g.device.type == "cpu"
        np.testing.assert_array_equal(g.numpy(), w.cpu().numpy())


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_to_host_vs_oracle_float64_output(pcf, prec):
    import torch
    s = synth.random_set(150, seed=72, max_len=60)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_pairwise_to_host(x, METRICS, precision=prec, out_dtype=torch.float64, bands=4)
    tol = 1e-12 if prec == "f64" else 1e-5
    for m, g in zip(METRICS, got):
        want = oracle.matrix(s, metric=m)
        diag = np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)]) if m == "gram" else None
        assert max_rel_error(m, g.numpy(), want, diag) <= tol, m


@pytest.mark.parametrize("n", [1, 5, 33, 64])
def test_to_host_small_sets(pcf, n):
    """Few tiles: AUTO takes the merge-path kernel (one walk, then one copy)."""
    s = synth.random_set(n, seed=73 + n, max_len=40)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    want = pcf.pcf_pairwise(x, METRICS, precision="f32c")
    got = pcf.pcf_pairwise_to_host(x, METRICS, precision="f32c")
    for w, g in zip(want, got):
        np.testing.assert_array_equal(g.numpy(), w.cpu().numpy())


def test_to_host_same_stream_and_given_buffers(pcf, stable700):
    """copy_stream = the compute stream (no overlap) and caller buffers; a
    second call overwrites them with the second set's matrices."""
    import torch
    s, x = stable700
    s2 = synth.PcfSet(s.offsets, s.times * 0.5, s.values[::-1].copy())
    x2 = pcf.PcfTensors.from_numpy(s2, "cuda")
    host = [torch.empty((s.n, s.n), dtype=torch.float32).pin_memory() for _ in METRICS]
    dev = [torch.empty((s.n, s.n), dtype=torch.float32, device="cuda") for _ in METRICS]
    cur = torch.cuda.current_stream()
    for xx in (x, x2):
        pcf.pcf_pairwise_to_host(xx, METRICS, precision="f32c", host_out=host, out=dev,
                                 bands=5, copy_stream=cur)
        want = pcf.pcf_pairwise(xx, METRICS, precision="f32c")
        for w, h in zip(want, host):
            np.testing.assert_array_equal(h.numpy(), w.cpu().numpy())


@pytest.mark.parametrize("bands", [0, 3, 16])
@pytest.mark.parametrize("schedule", ["tile512x2", "tile1024"])
def test_to_host_device_matrices_in_input_order(pcf, stable700, bands, schedule):
    """With a second copy stream the columns of the earlier bands' rows go
    back to the input order while the last band's rows are copied: the device
    matrices the call leaves behind equal pcf_pairwise's, bit for bit."""
    import torch
    s, x = stable700
    dev = [torch.full((s.n, s.n), float("nan"), dtype=torch.float32, device="cuda")
           for _ in METRICS]
    cs = torch.cuda.Stream()
    host = pcf.pcf_pairwise_to_host(x, METRICS, precision="f32c", out=dev, bands=bands,
                                    schedule=schedule, copy_stream=cs)
    torch.cuda.synchronize()
    want = pcf.pcf_pairwise(x, METRICS, precision="f32c", schedule=schedule)
    for w, d, h in zip(want, dev, host):
        np.testing.assert_array_equal(d.cpu().numpy(), w.cpu().numpy())
        np.testing.assert_array_equal(h.numpy(), w.cpu().numpy())


def test_to_host_rejects_pageable_buffers(pcf, stable700):
    import torch
    s, x = stable700
    with pytest.raises(ValueError):
        pcf.pcf_pairwise_to_host(x, ["l1"], host_out=[torch.empty((s.n, s.n))])


def test_to_host_reports_invalid_input(pcf):
    s = synth.random_set(100, seed=74, max_len=30)
    t = s.times.copy()
    k = int(s.offsets[40]) + 1
    t[k] = t[k - 1]
    x = pcf.PcfTensors.from_numpy(synth.PcfSet(s.offsets, t, s.values), "cuda")
    with pytest.raises(pcf.PcfError) as e:
        pcf.pcf_pairwise_to_host(x, ["l1"])
    assert e.value.index == k


def test_to_host_captured_in_cuda_graph(pcf, stable700):
    """The banded walk and the copies on the second stream are captured in one
    CUDA graph (the copy stream forks from and joins the capturing stream);
    replays after new input contents give the matrices of direct calls."""
    import torch
    s, x = stable700
    n = s.n
    host = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in METRICS]
    dev = [torch.empty((n, n), dtype=torch.float32, device="cuda") for _ in METRICS]
    ws = torch.empty(pcf.pcf_workspace_size(x, None, "f32c"), dtype=torch.uint8, device="cuda")
    copy = torch.cuda.Stream()

    def step():
        pcf.pcf_pairwise_to_host(x, METRICS, precision="f32c", host_out=host, out=dev,
                                 workspace=ws, bands=6, copy_stream=copy, check=False,
                                 schedule="tile512x3")

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for vals in (-s.values, s.values * 0.25):
        x.values.copy_(torch.from_numpy(np.ascontiguousarray(vals)))
        for h in host:
            h.zero_()
        g.replay()
        torch.cuda.synchronize()
        pcf.pcf_check(ws)
        want = pcf.pcf_pairwise(x, METRICS, precision="f32c", schedule="tile512x3")
        for w, h in zip(want, host):
            np.testing.assert_array_equal(h.numpy(), w.cpu().numpy())
    x.values.copy_(torch.from_numpy(np.ascontiguousarray(s.values)))


def test_to_host_full_size_sampled(pcf):
    """The benchmark's end-to-end configuration: N = 20,000 stable-rank PCFs,
    L1 + L2 + Gram, the default 16 bands, three 512-thread CTAs per SM.
    Sampled pairs against the oracle (the error measure of the device
    matrices), and sampled rows of every band equal to the device matrices."""
    import torch
    s = synth.stable_rank()
    n = s.n
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    dev = [torch.empty((n, n), dtype=torch.float32, device="cuda") for _ in METRICS]
    host = pcf.pcf_pairwise_to_host(x, METRICS, precision="f32c", out=dev, schedule="tile512x3")
    rng = np.random.default_rng(8)
    ii, jj = rng.integers(0, n, 200), rng.integers(0, n, 200)
    diag = {int(k): oracle.segment_sq(*s.pcf(int(k))) for k in np.concatenate([ii, jj])}
    for m, h in zip(METRICS, host):
        H = h.numpy()
        p = {"l1": 1.0, "l2": 2.0, "gram": 1.0}[m]
        for i, j in zip(ii, jj):
            I = oracle.integral(*s.pcf(int(i)), *s.pcf(int(j)), m, p)
            want = I if m == "gram" else brute.root(m, p, I)
            scale = (np.sqrt(diag[int(i)] * diag[int(j)]) if m == "gram" else abs(want)) or 1.0
            assert abs(float(H[i, j]) - want) / scale <= 1e-5, (m, i, j, H[i, j], want)
    rows = np.sort(rng.choice(n, 64, replace=False))
    for d, h in zip(dev, host):
        np.testing.assert_array_equal(h.numpy()[rows], d[torch.from_numpy(rows).cuda()].cpu().numpy())
