"""CUDA path vs the CPU oracle, element by element (needs a GPU).

Tolerances (per matrix, error measure of conftest.max_rel_error):
  float64 walk          <= 1e-12
  float32 compensated   <= 1e-5
  float32 plain         <= 5e-4
Dyadic inputs (small integers) are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_07183_gb300 import synth

from conftest import gpu_available, max_rel_error, read_golden

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32c": 1e-5, "f32b": 1e-5, "f32": 5e-4}


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


def _dev(P, s, dtype=None):
    return P.PcfTensors.from_numpy(s, "cuda", dtype=dtype)


def _gram_diag(s):
    return np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)])


def _metric_name(m):
    return m if isinstance(m, str) else m[0]


def _oracle(s, m, b=None):
    code = m if isinstance(m, str) else m[0]
    p = {"l1": 1.0, "l2": 2.0, "gram": 1.0}.get(code, None)
    root = True
    if isinstance(m, tuple):
        if code == "lp":
            p = float(m[1])
            root = m[2] if len(m) > 2 else True
        else:
            root = m[1]
    return oracle.matrix(s, b, metric=code, p=p, apply_root=root)


# --------------------------------------------------------------------------
def test_worked_example_sec5_2(pcf):
    g = read_golden("worked_example_sec5_2.txt")
    pcfs = [(g[f"pcf f{i}"][:, 0], g[f"pcf f{i}"][:, 1]) for i in range(1, 5)]
    offs = np.concatenate([[0], np.cumsum([len(t) for t, _ in pcfs])]).astype(np.int64)
    s = synth.PcfSet(offs, np.concatenate([t for t, _ in pcfs]),
                     np.concatenate([v for _, v in pcfs]))
    x = _dev(pcf, s)
    import torch
    for prec in ("f64", "f32c", "f32"):
        l1, gram, l35 = pcf.pcf_pairwise(x, ["l1", "gram", ("lp", 3.5)], precision=prec,
                                         out_dtype=torch.float64)
        np.testing.assert_array_equal(l1.cpu().numpy(), g["matrix l1 p=1"])
        np.testing.assert_array_equal(gram.cpu().numpy(), g["matrix gram p=1"])
        np.testing.assert_allclose(l35.cpu().numpy(), g["matrix lp p=3.5"], rtol=0,
                                   atol=6e-9 if prec == "f64" else 1e-5)


METRICS = ["l1", "l2", "gram", ("lp", 3.0), ("lp", 3.5), ("l2", False), ("lp", 2.5, False)]


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32b", "f32"])
@pytest.mark.parametrize("m", METRICS, ids=str)
def test_random_sets_vs_oracle(pcf, prec, m):
    import torch
    s = synth.random_set(150, seed=31, min_len=1, max_len=70)   # 5 blocks, ragged tail
    want = _oracle(s, m)
    got = pcf.pcf_pairwise(_dev(pcf, s), [m], precision=prec, out_dtype=torch.float64)[0]
    err = max_rel_error(_metric_name(m), got.cpu().numpy(), want, _gram_diag(s))
    assert err <= TOL[prec], (err, TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32b"])
@pytest.mark.parametrize("m", ["l1", "l2", "gram", ("lp", 3.0, False), ("l2", False)], ids=str)
def test_dyadic_bitwise(pcf, prec, m):
    """Integer gaps/values with many shared breakpoints: every integral is an
    exact integer, so the GPU must return the oracle's value exactly.  (Roots
    other than sqrt are compared with tolerance elsewhere: CUDA's pow and the
    host libm's pow may differ in the last bit.)"""
    import torch
    s = synth.dyadic(100, seed=41, max_len=40, min_len=1, max_gap=3, max_abs_value=8)
    want = _oracle(s, m)
    got = pcf.pcf_pairwise(_dev(pcf, s), [m], precision=prec, out_dtype=torch.float64)[0]
    np.testing.assert_array_equal(got.cpu().numpy(), want)


def test_dyadic_float32_plain_exact(pcf):
    import torch
    s = synth.dyadic(70, seed=42, max_len=30, max_gap=4, max_abs_value=6)
    for m in ("l1", "gram", ("l2", False)):
        got = pcf.pcf_pairwise(_dev(pcf, s, np.float32), [m], precision="f32",
                               out_dtype=torch.float64)[0]
        np.testing.assert_array_equal(got.cpu().numpy(), _oracle(s, m))


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_fused_equals_single(pcf, prec):
    import torch
    s = synth.random_set(90, seed=43, max_len=60)
    x = _dev(pcf, s)
    fused = pcf.pcf_pairwise(x, ["l1", "l2", "gram"], precision=prec, out_dtype=torch.float64)
    for m, f in zip(["l1", "l2", "gram"], fused):
        single = pcf.pcf_pairwise(x, [m], precision=prec, out_dtype=torch.float64)[0]
        np.testing.assert_array_equal(f.cpu().numpy(), single.cpu().numpy())
    fused = pcf.pcf_pairwise(x, [("lp", 3.0), "l2", "l1"], precision=prec, out_dtype=torch.float64)
    for m, f in zip([("lp", 3.0), "l2", "l1"], fused):
        err = max_rel_error(_metric_name(m), f.cpu().numpy(), _oracle(s, m), None)
        assert err <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_upper_packed_layout(pcf, prec):
    import torch
    s = synth.random_set(77, seed=44, max_len=50)
    x = _dev(pcf, s)
    full = pcf.pcf_pairwise(x, ["l1", "gram"], precision=prec, out_dtype=torch.float32)
    up = pcf.pcf_pairwise(x, ["l1", "gram"], precision=prec, layout="upper",
                          out_dtype=torch.float32)
    iu = np.triu_indices(s.n)
    for f, u in zip(full, up):
        f = f.cpu().numpy()
        np.testing.assert_array_equal(f, f.T)
        np.testing.assert_array_equal(u.cpu().numpy(), f[iu])


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32b"])
def test_long_pcfs_use_several_windows(pcf, prec):
    """Lengths well beyond one shared-memory window (about 450 float32 or 220
    float64 elements per PCF) so that the time-window staging is exercised."""
    import torch
    rng = np.random.default_rng(5)
    lens = np.concatenate([rng.integers(2, 40, 40), rng.integers(300, 2500, 30)])
    s = synth.from_lengths(lens, lambda r, m: r.exponential(1.0, m),
                           lambda r, o: np.where(np.isin(np.arange(o[-1]), o[1:] - 1), 0.0,
                                                 r.standard_normal(o[-1])),
                           rng, np.float64, "long")
    x = _dev(pcf, s)
    got = pcf.pcf_pairwise(x, ["l1", "l2", "gram"], precision=prec, out_dtype=torch.float64)
    for m, g in zip(["l1", "l2", "gram"], got):
        err = max_rel_error(m, g.cpu().numpy(), _oracle(s, m), _gram_diag(s))
        assert err <= TOL[prec], (m, err)


def test_long_dyadic_windows_bitwise(pcf):
    import torch
    s = synth.dyadic(40, seed=45, max_len=1500, min_len=200, max_gap=2, max_abs_value=4)
    got = pcf.pcf_pairwise(_dev(pcf, s), ["l1", ("l2", False), "gram"], precision="f64",
                           out_dtype=torch.float64)
    for m, g in zip(["l1", ("l2", False), "gram"], got):
        np.testing.assert_array_equal(g.cpu().numpy(), _oracle(s, m))


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_cross_blocks(pcf, prec):
    import torch
    a = synth.random_set(70, seed=46, max_len=60)
    b = synth.random_set(45, seed=47, max_len=90)
    xa, xb = _dev(pcf, a), _dev(pcf, b)
    want = {m: _oracle(a, m, b) for m in ("l1", "l2", ("lp", 3.0))}
    out = torch.full((a.n, b.n + 3), np.nan, dtype=torch.float64, device="cuda")
    outs = [out.clone() for _ in range(3)]
    for r0 in range(0, a.n, 32):
        r1 = min(a.n, r0 + 32)
        views = [o[r0:r1] for o in outs]
        pcf.pcf_cross(xa, xb, r0, r1, ["l1", "l2", ("lp", 3.0)], precision=prec,
                      out=views, ld_out=b.n + 3, reuse_b=r0 > 0)
    for m, o in zip(("l1", "l2", ("lp", 3.0)), outs):
        o = o.cpu().numpy()
        assert np.all(np.isnan(o[:, b.n:]))
        err = max_rel_error(_metric_name(m), o[:, :b.n], want[m])
        assert err <= TOL[prec], (m, err)


def test_edge_cases(pcf):
    import torch
    # N = 1, length-1 PCFs, duplicates, non-zero tails (divergent integrals)
    pcfs = [([0.0], [0.0]), ([0.0], [2.0]), ([0.0, 1.0], [3.0, 2.0]),
            ([0.0, 1.0, 4.0], [1.0, -1.0, 0.0]), ([0.0, 1.0, 4.0], [1.0, -1.0, 0.0])]
    offs = np.concatenate([[0], np.cumsum([len(t) for t, _ in pcfs])]).astype(np.int64)
    s = synth.PcfSet(offs, np.concatenate([t for t, _ in pcfs]).astype(np.float64),
                     np.concatenate([v for _, v in pcfs]).astype(np.float64))
    x = _dev(pcf, s)
    for prec in ("f64", "f32c", "f32"):
        for m in ("l1", "l2", "gram", ("lp", 3.5)):
            got = pcf.pcf_pairwise(x, [m], precision=prec, out_dtype=torch.float64)[0].cpu().numpy()
            want = _oracle(s, m)
            np.testing.assert_array_equal(np.isinf(got), np.isinf(want))
            np.testing.assert_array_equal(np.sign(got), np.sign(want))
            fin = np.isfinite(want)
            np.testing.assert_allclose(got[fin], want[fin], rtol=1e-6)
    one = synth.PcfSet(np.array([0, 3]), np.array([0.0, 1.0, 2.0]), np.array([1.0, 2.0, 0.0]))
    g = pcf.pcf_pairwise(_dev(pcf, one), ["gram", "l1"], precision="f64", out_dtype=torch.float64)
    assert g[0].item() == 5.0 and g[1].item() == 0.0


@pytest.mark.parametrize("case,detail", [("t0", 2), ("order", 3), ("nan_t", 4),
                                          ("nan_v", 5), ("offsets", 1), ("range32", 6)])
def test_invalid_input_is_reported(pcf, case, detail):
    s = synth.random_set(40, seed=48, min_len=3, max_len=10)
    t, v, o = s.times.copy(), s.values.copy(), s.offsets.copy()
    k = int(o[7]) + 1
    if case == "t0":
        t[o[5]] = 0.25
    elif case == "order":
        t[k + 1] = t[k]
    elif case == "nan_t":
        t[k] = np.nan
    elif case == "nan_v":
        v[k] = np.inf
    elif case == "offsets":
        o[9] = o[10] + 1
    elif case == "range32":
        t[int(o[40]) - 1] = 1e300
    x = _dev(pcf, synth.PcfSet(o, t, v))
    prec = "f32c" if case == "range32" else "f64"
    with pytest.raises(pcf.PcfError) as ei:
        pcf.pcf_pairwise(x, ["l1"], precision=prec)
    assert ei.value.detail == detail


def test_float32_input_all_precisions(pcf):
    import torch
    s = synth.lognormal(400, max_len=1200)
    x = _dev(pcf, s)
    want = _oracle(s, "gram")
    for prec in ("f64", "f32c", "f32b", "f32"):
        got = pcf.pcf_pairwise(x, ["gram"], precision=prec, out_dtype=torch.float64)[0]
        err = max_rel_error("gram", got.cpu().numpy(), want, _gram_diag(s))
        assert err <= TOL[prec], (prec, err)


# --------------------------------------------------------------------------
# Full-size workloads: sampled pairs against the oracle one by one
# --------------------------------------------------------------------------
def _sampled_check(s, mats, metrics, prec, npairs, seed, layout="full", gram_diag=None):
    rng = np.random.default_rng(seed)
    N = s.n
    ii = rng.integers(0, N, npairs)
    jj = rng.integers(0, N, npairs)
    for m, M in zip(metrics, mats):
        name = _metric_name(m)
        code = name
        p = {"l1": 1.0, "l2": 2.0, "gram": 1.0}.get(name, None)
        if name == "lp":
            p = float(m[1])
        for i, j in zip(ii, jj):
            I = oracle.integral(*s.pcf(i), *s.pcf(j), code, p)
            want = brute.root(code, p, I) if name != "gram" else I
            if layout == "full":
                got = float(M[i, j])
            else:
                lo, hi = min(i, j), max(i, j)
                got = float(M[lo * N - lo * (lo - 1) // 2 + (hi - lo)])
            if name == "gram":
                scale = np.sqrt(gram_diag[i] * gram_diag[j]) or 1.0
            else:
                scale = abs(want) or 1.0
            assert abs(got - want) / scale <= TOL[prec], (name, i, j, got, want)


def test_lognormal_sampled_upper_packed(pcf):
    """Uneven log-normal lengths (up to 10,000 points), float32 Gram, packed
    upper triangle; N = 30,000 keeps the test's output at 1.8 GB."""
    import torch
    s = synth.lognormal(30000)
    x = _dev(pcf, s)
    M = pcf.pcf_pairwise(x, ["gram"], precision="f32c", layout="upper",
                         out_dtype=torch.float32)[0].cpu().numpy()
    diag = np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)])
    _sampled_check(s, [M], ["gram"], "f32c", 300, 8, layout="upper", gram_diag=diag)


def test_cuda_graph_replay_with_new_contents(pcf):
    """One captured graph, replayed after new PCF contents of the same shape
    are copied into the input tensors."""
    import torch
    a = synth.random_set(80, seed=61, min_len=3, max_len=30)
    b = synth.PcfSet(a.offsets, a.times * 2.0, -a.values)
    x = _dev(pcf, a)
    g = pcf.PairwiseGraph(x, ["l1", "gram"], precision="f64", out_dtype=torch.float64)
    for s in (a, b, a):
        x.times.copy_(torch.from_numpy(s.times))
        x.values.copy_(torch.from_numpy(s.values))
        l1, gram = [o.clone() for o in g.replay()]
        g.check()
        assert max_rel_error("l1", l1.cpu().numpy(), _oracle(s, "l1")) <= 1e-12
        assert max_rel_error("gram", gram.cpu().numpy(), _oracle(s, "gram"), _gram_diag(s)) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_cross_streamed_to_host(pcf, prec):
    """Row blocks double-buffered on the device and copied to pinned host
    memory; the host result is the whole cross matrix."""
    import torch
    a = synth.random_set(131, seed=62, max_len=70)
    b = synth.random_set(57, seed=63, max_len=90)
    xa, xb = _dev(pcf, a), _dev(pcf, b)
    host = pcf.pcf_cross_to_host(xa, xb, ["l1", "gram"], precision=prec, block_rows=40,
                                 out_dtype=torch.float64)
    assert host[0].is_pinned()
    for m, h in zip(("l1", "gram"), host):
        want = _oracle(a, m, b)
        if m == "gram":
            da = np.array([oracle.segment_sq(*a.pcf(i)) for i in range(a.n)])
            db = np.array([oracle.segment_sq(*b.pcf(j)) for j in range(b.n)])
            scale = np.sqrt(np.outer(da, db))
            err = np.max(np.abs(h.numpy() - want) / np.where(scale > 0, scale, 1.0))
        else:
            err = max_rel_error(m, h.numpy(), want)
        assert err <= TOL[prec], (m, err)


@pytest.mark.parametrize("sched", ["tile1024", "tile512x2", "mergepath"])
def test_sorted_output_layout(pcf, sched):
    """Layout "sorted": entry (s, t) is F of the s-th and t-th PCFs of the
    library's sort order, bit-identical to the full layout permuted."""
    import torch
    rng = np.random.default_rng(64)
    lens = np.concatenate([rng.integers(1, 80, 90), rng.integers(257, 400, 10)])
    s = synth.from_lengths(lens, lambda r, m: r.exponential(1.0, m),
                           lambda r, o: np.where(np.isin(np.arange(o[-1]), o[1:] - 1), 0.0,
                                                 r.standard_normal(o[-1])),
                           rng, np.float64, "mixed")
    x = _dev(pcf, s)
    ws = pcf.pcf_prepare(x, "f64")
    srt = pcf.pcf_pairwise(x, ["l1", "gram"], precision="f64", layout="sorted", workspace=ws,
                           prepared=True, out_dtype=torch.float64, schedule=sched)
    perm = pcf.pcf_sort_order(x, ws, "f64").cpu().numpy().astype(np.int64)
    assert sorted(perm.tolist()) == list(range(s.n))
    from paper_2404_07183_gb300 import shard
    np.testing.assert_array_equal(perm, shard.sorted_order(s.lengths(), s.times[s.offsets[1:] - 1]))
    full = pcf.pcf_pairwise(x, ["l1", "gram"], precision="f64", out_dtype=torch.float64,
                            schedule=sched)
    for a_, b_ in zip(srt, full):
        np.testing.assert_array_equal(a_.cpu().numpy(), b_.cpu().numpy()[np.ix_(perm, perm)])
