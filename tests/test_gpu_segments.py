"""Segment iteration on the GPU (single-PCF integrals over [a, b]) against
the oracle (needs a GPU)."""
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


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("kind,p,root", [("integral", 1.0, False), ("lp", 1.0, False),
                                         ("lp", 2.0, True), ("lp", 3.0, False),
                                         ("lp", 3.5, True)])
@pytest.mark.parametrize("ab", [(0.0, np.inf), (0.5, 7.25), (3.0, 1e9)])
def test_segments_vs_oracle(pcf, prec, dtype, kind, p, root, ab):
    import torch
    s = synth.random_set(300, seed=101, min_len=1, max_len=90).astype(dtype)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    got = pcf.pcf_segment_integrals(x, kind, p, root, ab[0], ab[1], precision=prec).cpu().numpy()
    if prec == "f32c" and dtype == np.float64:
        s = s.astype(np.float32)      # the float32 walk sees the rounded input
    for i in range(s.n):
        t, v = s.pcf(i)
        want = oracle.segment_integral(t, v, kind, p, ab[0], ab[1])
        if root and kind == "lp" and np.isfinite(want):
            want = want ** (1.0 / p)
        if np.isinf(want):
            assert got[i] == want
        elif prec == "f64":
            assert abs(got[i] - want) <= 1e-12 * max(1.0, abs(want)), (i, got[i], want)
        else:
            # float32 terms carry a few ulp each: bound by int |h| (its root for norms)
            scale = oracle.segment_integral(t, v, "lp", 1.0 if kind == "integral" else p,
                                            ab[0], ab[1])
            if root and kind == "lp":
                scale = scale ** (1.0 / p)
            assert abs(got[i] - want) <= 1e-5 * scale + 1e-30, (i, got[i], want)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_segments_dyadic_exact_and_edges(pcf, prec):
    s = synth.dyadic(200, seed=102, max_len=50, min_len=1, final_zero=False)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for kind, p in (("integral", 1.0), ("lp", 2.0)):
        got = pcf.pcf_segment_integrals(x, kind, p, False, 2.0, 40.0,
                                        precision=prec).cpu().numpy()
        want = np.array([oracle.segment_integral(*s.pcf(i), kind, p, 2.0, 40.0)
                         for i in range(s.n)])
        np.testing.assert_array_equal(got, want)
        tail = pcf.pcf_segment_integrals(x, kind, p, precision=prec).cpu().numpy()
        want = np.array([oracle.segment_integral(*s.pcf(i), kind, p) for i in range(s.n)])
        np.testing.assert_array_equal(tail, want)     # +-inf where the last value != 0


def test_segments_norm_matches_gram_diagonal(pcf):
    import torch
    s = synth.stable_rank(500, seed=103)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    sq = pcf.pcf_segment_integrals(x, "lp", 2.0).cpu().numpy()
    gram = pcf.pcf_pairwise(x, ["gram"], precision="f64", out_dtype=torch.float64)[0]
    np.testing.assert_allclose(np.diag(gram.cpu().numpy()), sq, rtol=1e-13)


def test_segments_reject_bad_arguments(pcf):
    s = synth.random_set(5, seed=104)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    with pytest.raises(pcf.PcfError):
        pcf.pcf_segment_integrals(x, "lp", 0.5)
    with pytest.raises(pcf.PcfError):
        pcf.pcf_segment_integrals(x, "lp", 2.0, a=3.0, b=1.0)
    with pytest.raises(pcf.PcfError):
        pcf.pcf_segment_integrals(x, "lp", 2.0, precision="f32")
    t = s.times.copy()
    t[3] = t[2]
    bad = pcf.PcfTensors.from_numpy(synth.PcfSet(s.offsets, t, s.values), "cuda")
    with pytest.raises(pcf.PcfError):
        pcf.pcf_segment_integrals(bad, "integral")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_segments_long_pcfs(pcf, prec):
    """PCFs of 1,000 to 5,000 breakpoints among short ones: PCFs that run
    past the end of the chunk that owns them."""
    a = synth.random_set(12, seed=105, min_len=1000, max_len=5000)
    b = synth.random_set(60, seed=106, min_len=1, max_len=200)
    s = synth.PcfSet(np.concatenate([b.offsets, b.offsets[-1] + a.offsets[1:]]),
                     np.concatenate([b.times, a.times]), np.concatenate([b.values, a.values]))
    s = synth.subset(s, np.random.default_rng(7).permutation(s.n))
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    for kind, p, root, ab in (("lp", 2.0, True, (0.0, np.inf)), ("integral", 1.0, False, (1.5, 40.0)),
                              ("lp", 3.5, False, (0.0, 25.0))):
        got = pcf.pcf_segment_integrals(x, kind, p, root, ab[0], ab[1], precision=prec).cpu().numpy()
        for i in range(s.n):
            t, v = s.pcf(i)
            want = oracle.segment_integral(t, v, kind, p, ab[0], ab[1])
            scale = oracle.segment_integral(t, v, "lp", 1.0 if kind == "integral" else p, ab[0], ab[1])
            if root and kind == "lp":
                want, scale = want ** (1.0 / p), scale ** (1.0 / p)
            tol = 1e-12 if prec == "f64" else 1e-5
            assert abs(got[i] - want) <= tol * scale + 1e-30, (i, s.lengths()[i], got[i], want)


def test_segments_error_report_matches_pairwise_check(pcf):
    """The check inside the segment kernels reports what pcf_pairwise's does:
    here the smallest offending element lies in a long PCF."""
    a = synth.random_set(3, seed=107, min_len=2000, max_len=3000)
    b = synth.random_set(20, seed=108, min_len=5, max_len=50)
    s = synth.PcfSet(np.concatenate([a.offsets, a.offsets[-1] + b.offsets[1:]]),
                     np.concatenate([a.times, b.times]), np.concatenate([a.values, b.values]))
    t, v = s.times.copy(), s.values.copy()
    k_long = int(s.offsets[1]) + 1500            # inside PCF 1 (long)
    k_short = int(s.offsets[10]) + 3             # inside a short PCF, larger index
    v[k_long] = np.nan
    t[k_short] = t[k_short - 1]
    bad = pcf.PcfTensors.from_numpy(synth.PcfSet(s.offsets, t, v), "cuda")
    with pytest.raises(pcf.PcfError) as e1:
        pcf.pcf_segment_integrals(bad, "lp", 2.0)
    with pytest.raises(pcf.PcfError) as e2:
        pcf.pcf_pairwise(bad, ["l1"])
    assert (e1.value.detail, e1.value.index) == (e2.value.detail, e2.value.index) == (5, k_long)
    # a time that is not finite in a long PCF, offsets error elsewhere: offsets first
    off = s.offsets.copy()
    off[15] = off[14]
    bad2 = pcf.PcfTensors.from_numpy(synth.PcfSet(off, t, s.values), "cuda")
    with pytest.raises(pcf.PcfError) as e1:
        pcf.pcf_segment_integrals(bad2, "integral", precision="f32c")
    with pytest.raises(pcf.PcfError) as e2:
        pcf.pcf_pairwise(bad2, ["l1"], precision="f32c")
    assert (e1.value.detail, e1.value.index) == (e2.value.detail, e2.value.index) == (1, 14)


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_segments_full_size_sampled(pcf, prec):
    """The benchmarked workload (log-normal N = 100,000, lengths up to ~10^4),
    checked on every 97th PCF against the oracle."""
    s = synth.lognormal()
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    norm = pcf.pcf_segment_integrals(x, "lp", 2.0, True, precision=prec).cpu().numpy()
    integ = pcf.pcf_segment_integrals(x, "integral", precision=prec).cpu().numpy()
    tol = 1e-12 if prec == "f64" else 1e-5
    for i in range(0, s.n, 97):
        t, v = s.pcf(i)
        want = oracle.segment_integral(t, v, "lp", 2.0) ** 0.5
        assert abs(norm[i] - want) <= tol * want + 1e-30, (i, norm[i], want)
        w = oracle.segment_integral(t, v, "integral")
        scale = oracle.segment_integral(t, v, "lp", 1.0)
        assert abs(integ[i] - w) <= tol * scale + 1e-30, (i, integ[i], w)


def _mixed_layout_set(seed):
    """Lengths chosen to cross every boundary of the flat pass: thousands of
    length-1 and length-2 PCFs (several staged batches of PCF offsets inside
    one 7,680-breakpoint chunk), PCFs of 20,000 and 41,000 breakpoints (many
    rounds, several chunks, no PCF starting in some chunks), and random
    lengths with an odd total."""
    rng = np.random.default_rng(seed)
    parts = [synth.random_set(1500, seed=seed + 1, min_len=1, max_len=2),
             synth.random_set(1, seed=seed + 2, min_len=20000, max_len=20000),
             synth.random_set(300, seed=seed + 3, min_len=1, max_len=300),
             synth.random_set(1, seed=seed + 4, min_len=41000, max_len=41000),
             synth.random_set(1200, seed=seed + 5, min_len=1, max_len=3),
             synth.random_set(77, seed=seed + 6, min_len=2000, max_len=9000)]
    offs, ts, vs, base = [np.zeros(1, np.int64)], [], [], 0
    for p in parts:
        offs.append(p.offsets[1:] + base)
        base += int(p.offsets[-1])
        ts.append(p.times)
        vs.append(p.values)
    s = synth.PcfSet(np.concatenate(offs), np.concatenate(ts), np.concatenate(vs))
    return synth.subset(s, rng.permutation(s.n)) if seed % 2 else s


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("aligned", [True, False])
def test_segments_chunk_and_batch_layouts(pcf, prec, dtype, aligned):
    """Every PCF of a set whose lengths cross the chunk, round and batch
    boundaries of the flat pass, with 16-byte aligned arrays (vector loads)
    and with arrays that start one element off (scalar loads)."""
    import torch
    s = _mixed_layout_set(11 if aligned else 12).astype(dtype)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    if not aligned:
        def shifted(a):
            big = torch.empty(a.numel() + 1, dtype=a.dtype, device=a.device)
            big[1:] = a
            return big[1:]
        x = pcf.PcfTensors(x.offsets, shifted(x.times), shifted(x.values))
        assert x.times.data_ptr() % 16 != 0
    # float64 data integrated in float32: the oracle sees the rounded input
    ref = s.astype(np.float32) if (prec == "f32c" and dtype == np.float64) else s
    tol = 1e-12 if prec == "f64" else 1e-5
    for kind, p, root, ab in (("lp", 2.0, True, (0.0, np.inf)),
                              ("integral", 1.0, False, (0.75, 60.0))):
        got = pcf.pcf_segment_integrals(x, kind, p, root, ab[0], ab[1],
                                        precision=prec).cpu().numpy()
        for i in range(s.n):
            t, v = ref.pcf(i)
            want = oracle.segment_integral(t, v, kind, p, ab[0], ab[1])
            scale = oracle.segment_integral(t, v, "lp", 1.0 if kind == "integral" else p,
                                            ab[0], ab[1])
            if root:
                want, scale = want ** (1.0 / p), scale ** (1.0 / p)
            if np.isinf(want):
                assert got[i] == want, (i, got[i], want)
            else:
                assert abs(got[i] - want) <= tol * scale + 1e-30, (i, s.lengths()[i], got[i], want)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("lengths", [[16] * 1024, [4096] * 5 + [1] * 3, [8192] * 3 + [8191, 1],
                                     [7680] * 3 + [7679, 1], [3840] * 6 + [2048] * 3,
                                     [1] * 8192 + [16] * 512, [8193, 4095, 1, 16, 15, 17] * 3])
def test_segments_boundaries_on_thread_round_chunk_edges(pcf, prec, lengths):
    """PCF boundaries exactly on the 16-breakpoint thread ranges, the
    4,096-breakpoint rounds and the 7,680-breakpoint chunks of the flat pass
    (and one off), float32 data (vector loads)."""
    rng = np.random.default_rng(sum(lengths) % 1000)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    t = np.empty(offs[-1]); v = np.empty(offs[-1])
    for i, n in enumerate(lengths):
        g = rng.exponential(1.0, n - 1)
        t[offs[i]:offs[i + 1]] = np.concatenate([[0.0], np.cumsum(g)])
        vv = rng.standard_normal(n)
        vv[-1] = 0.0
        v[offs[i]:offs[i + 1]] = vv
    s = synth.PcfSet(offs, t, v).astype(np.float32)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    tol = 1e-12 if prec == "f64" else 1e-5
    for kind, p, root in (("lp", 2.0, True), ("integral", 1.0, False)):
        got = pcf.pcf_segment_integrals(x, kind, p, root, precision=prec).cpu().numpy()
        for i in range(s.n):
            ti, vi = s.pcf(i)
            want = oracle.segment_integral(ti, vi, kind, p)
            scale = oracle.segment_integral(ti, vi, "lp", 1.0 if kind == "integral" else p)
            if root:
                want, scale = want ** (1.0 / p), scale ** (1.0 / p)
            assert abs(got[i] - want) <= tol * scale + 1e-30, (i, lengths[i], got[i], want)


def _set_from_lengths(lengths, seed, dtype=np.float64):
    """PCFs with the given lengths: times 0, g_1, g_1 + g_2, ... (gaps
    uniform in [0.5, 1.5]), values N(0, 1) with the last one 0."""
    rng = np.random.default_rng(seed)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    t = np.empty(offs[-1]); v = np.empty(offs[-1])
    for i, n in enumerate(lengths):
        t[offs[i]:offs[i + 1]] = np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, n - 1))])
        vv = rng.standard_normal(n)
        vv[-1] = 0.0
        v[offs[i]:offs[i + 1]] = vv
    return synth.PcfSet(offs, t, v).astype(dtype)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("lengths", [
    [5, 100_000, 7],                          # one long PCF, several chunks
    [40_000, 35_000, 3, 61_441],              # long PCFs back to back (a chunk with two pieces)
    [7680 - 17, 7680 * 5, 17, 7680 * 4 + 1],  # long PCFs starting / ending on chunk edges
    [30_720, 30_721, 2],                      # at and just above the long threshold
    [100, 7680 * 5 - 100],                    # long last PCF, breakpoint count a multiple of the chunk
    [7680 * 5, 7680 * 5],                     # a long PCF ending exactly on a chunk edge
    [31_000],                                 # a single long PCF
])
def test_segments_long_pcfs_split_into_pieces(pcf, prec, dtype, lengths):
    """PCFs longer than four 7,680-breakpoint chunks are split at the chunk
    edges, integrated one piece per CTA and combined in piece order."""
    s = _set_from_lengths(lengths, seed=len(lengths) + sum(lengths) % 97, dtype=dtype)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    tol = 1e-12 if prec == "f64" else 1e-5
    for kind, p, root, ab in (("lp", 2.0, True, (0.0, np.inf)), ("integral", 1.0, False, (0.0, np.inf)),
                              ("lp", 1.0, False, (2.5, 31_000.0))):
        got = pcf.pcf_segment_integrals(x, kind, p, root, ab[0], ab[1], precision=prec).cpu().numpy()
        for i in range(s.n):
            ti, vi = s.pcf(i)
            want = oracle.segment_integral(ti, vi, kind, p, ab[0], ab[1])
            scale = oracle.segment_integral(ti, vi, "lp", 1.0 if kind == "integral" else p, ab[0], ab[1])
            if root:
                want, scale = want ** (1.0 / p), scale ** (1.0 / p)
            assert abs(got[i] - want) <= tol * scale + 1e-30, (i, lengths[i], got[i], want)


def test_segments_long_pcf_repeatable_and_error_report(pcf):
    """The pieces of a long PCF are summed in a fixed order (same bits on a
    second call); an invalid breakpoint in a later piece is reported as by
    pcf_pairwise's check."""
    s = _set_from_lengths([3, 90_000, 4], seed=5, dtype=np.float32)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    a1 = pcf.pcf_segment_integrals(x, "lp", 2.0, True, precision="f32c").cpu().numpy()
    a2 = pcf.pcf_segment_integrals(x, "lp", 2.0, True, precision="f32c").cpu().numpy()
    np.testing.assert_array_equal(a1, a2)
    t, v = s.times.copy(), s.values.copy()
    k = int(s.offsets[1]) + 70_001            # in the tenth piece of the long PCF
    v[k] = np.inf
    t[k + 5] = t[k + 4]                       # and an order error after it
    bad = pcf.PcfTensors.from_numpy(synth.PcfSet(s.offsets, t, v), "cuda")
    with pytest.raises(pcf.PcfError) as e1:
        pcf.pcf_segment_integrals(bad, "integral", precision="f32c")
    with pytest.raises(pcf.PcfError) as e2:
        pcf.pcf_pairwise(bad, ["l1"], precision="f32c")
    assert (e1.value.detail, e1.value.index) == (e2.value.detail, e2.value.index) == (5, k)


def test_segments_long_pcfs_in_cuda_graph(pcf):
    """The piece grid is a programmatic dependent of the main pass; captured in
    a CUDA graph and replayed with new contents, the results equal those of
    direct calls bit for bit, for both functionals back to back."""
    import torch
    s = _set_from_lengths([5, 100_000, 7, 40_000, 300], seed=11, dtype=np.float32)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    ws = torch.empty(pcf.pcf_workspace_size(x, None, "f64"), dtype=torch.uint8, device="cuda")
    o1 = torch.empty(s.n, dtype=torch.float64, device="cuda")
    o2 = torch.empty(s.n, dtype=torch.float64, device="cuda")

    def step():
        pcf.pcf_segment_integrals(x, "lp", 2.0, True, precision="f32c", out=o1, workspace=ws,
                                  check=False)
        pcf.pcf_segment_integrals(x, "integral", precision="f32c", out=o2, workspace=ws,
                                  check=False)

    step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for vals in (s.values, -2.0 * s.values, s.values):
        x.values.copy_(torch.from_numpy(np.ascontiguousarray(vals)))
        g.replay()
        torch.cuda.synchronize()
        pcf.pcf_check(ws)
        r1, r2 = o1.cpu().numpy(), o2.cpu().numpy()
        step()
        np.testing.assert_array_equal(r1, o1.cpu().numpy())
        np.testing.assert_array_equal(r2, o2.cpu().numpy())
        for i in range(s.n):
            ti, vi = s.pcf(i)
            vi = vals[s.offsets[i]:s.offsets[i + 1]].astype(np.float64)
            want = oracle.segment_integral(ti, vi, "lp", 2.0) ** 0.5
            assert abs(r1[i] - want) <= 1e-5 * want + 1e-30, (i, r1[i], want)
            want = oracle.segment_integral(ti, vi, "integral", 1.0)
            scale = oracle.segment_integral(ti, vi, "lp", 1.0)
            assert abs(r2[i] - want) <= 1e-5 * scale + 1e-30, (i, r2[i], want)
