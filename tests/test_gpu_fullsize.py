"""The benchmarked workloads at their full sizes, against the oracle (needs a GPU).

Each workload runs in the configuration the benchmark times; outputs too
large to compare whole are checked on sampled entries, each recomputed by the
oracle's float64 walk (gathered on the device, so only the samples travel).
Tolerances are the per-matrix targets: float64 <= 1e-12, compensated float32
<= 1e-5 (distances relative to the entry, Gram against sqrt(G*_ii G*_jj)).

  uniform N = 1,000 (L1)            every pair, all precisions
  stable-rank N = 20,000            L1 + L2 + Gram fused; float64 walk at
                                    float64 output, compensated float32 walks
  log-normal N = 100,000            Gram, packed upper triangle (5.0e9 entries:
                                    packed indices beyond 2^32 are sampled)
  Euler 50,000 x 50,000 cross       L1 + L2 + L3 fused (compensated float32),
                                    streamed to host memory, on a row block
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_07183_gb300 import synth

from conftest import gpu_available, max_rel_error

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32c": 1e-5, "f32b": 1e-5, "f32": 5e-4}


@pytest.fixture(scope="module")
def pcf():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import paper_2404_07183_gb300 as P
    P.build.build()
    return P


def _want(s, i, j, name, p, b=None):
    tb, vb = (b if b is not None else s).pcf(j)
    I = oracle.integral(*s.pcf(i), tb, vb, name, p)
    return I if name == "gram" else brute.root(name, p, I)


def _scale(s, i, j, name, want, b=None):
    if name == "gram":
        gi = oracle.segment_sq(*s.pcf(i))
        gj = oracle.segment_sq(*(b if b is not None else s).pcf(j))
        return np.sqrt(gi * gj) or 1.0
    return abs(want) or 1.0


def _check_entries(s, got, ii, jj, name, p, tol, b=None):
    worst = 0.0
    for g, i, j in zip(got, ii, jj):
        w = _want(s, int(i), int(j), name, p, b)
        if w == 0.0:
            assert g == 0.0, (name, i, j, g)
            continue
        e = abs(float(g) - w) / _scale(s, int(i), int(j), name, w, b)
        worst = max(worst, e)
        assert e <= tol, (name, int(i), int(j), float(g), w, e)
    return worst


@pytest.mark.parametrize("prec", ["f64", "f32c", "f32b"])
def test_uniform_n1000_every_pair(pcf, prec):
    """N = 1,000, n ~ U{10..100}: the whole L1 matrix against the oracle's."""
    import torch
    s = synth.uniform_small()
    got = pcf.pcf_pairwise(pcf.PcfTensors.from_numpy(s, "cuda"), ["l1"], precision=prec,
                           out_dtype=torch.float64)[0].cpu().numpy()
    want = oracle.matrix(s, metric="l1")
    assert max_rel_error("l1", got, want) <= TOL[prec]
    np.testing.assert_array_equal(got, got.T)


@pytest.mark.parametrize("prec,out_dtype", [("f64", "f64"), ("f32c", "f32"), ("f32b", "f32")])
def test_stable_rank_n20000_sampled(pcf, prec, out_dtype):
    """N = 20,000 stable-rank curves, L1 + L2 + Gram in one walk; 1,000 sampled
    pairs per matrix.  The float64 walk is read at float64 output against the
    float64 target; the float32 walks at float32 output."""
    import torch
    s = synth.stable_rank()
    od = torch.float64 if out_dtype == "f64" else torch.float32
    mats = pcf.pcf_pairwise(pcf.PcfTensors.from_numpy(s, "cuda"), ["l1", "l2", "gram"],
                            precision=prec, out_dtype=od)
    rng = np.random.default_rng(17)
    ii = rng.integers(0, s.n, 1000)
    jj = rng.integers(0, s.n, 1000)
    ti, tj = torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()
    for name, p, M in zip(("l1", "l2", "gram"), (1.0, 2.0, 1.0), mats):
        got = M[ti, tj].double().cpu().numpy()
        _check_entries(s, got, ii, jj, name, p, TOL[prec])
        d = torch.diagonal(M).double().cpu().numpy()
        if name != "gram":
            assert np.all(d == 0.0)


def test_lognormal_n100000_upper_packed(pcf):
    """The configured uneven workload: N = 100,000, log-normal lengths (up to
    10,000 points), float32, Gram in the packed upper triangle.  The packed
    matrix has 5.0e9 entries, so its indices pass 2^32; half of the sampled
    pairs lie beyond that point."""
    import torch
    s = synth.lognormal()
    N = s.n
    M = pcf.pcf_pairwise(pcf.PcfTensors.from_numpy(s, "cuda"), ["gram"], precision="f32c",
                         layout="upper", out_dtype=torch.float32)[0]
    assert M.numel() == N * (N + 1) // 2
    rng = np.random.default_rng(18)
    # rows r with r * N - r (r - 1) / 2 > 2^32 start near r = 48,000
    first_row_past = int(np.argmax([r * N - r * (r - 1) // 2 > 2 ** 32 for r in range(N)]))
    lo = np.concatenate([rng.integers(0, first_row_past, 500),
                         rng.integers(first_row_past, N, 500)])
    hi = np.array([int(rng.integers(l, N)) for l in lo])
    idx = lo * N - lo * (lo - 1) // 2 + (hi - lo)
    assert np.sum(idx > 2 ** 32) >= 500
    got = M[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    _check_entries(s, got, lo, hi, "gram", 1.0, TOL["f32c"])


def test_euler_cross_row_block_to_host(pcf):
    """Euler-curve cross matrix (n = 1,000, integer walk values, float32):
    L1 + L2 + L3 fused in one compensated float32 walk, block-streamed to
    pinned host memory, for 2,048 rows of A against all 50,000 PCFs of B;
    1,000 sampled entries per matrix against the oracle."""
    import torch
    A, B = synth.euler()
    rows = synth.subset(A, np.arange(20000, 22048))
    xa = pcf.PcfTensors.from_numpy(rows, "cuda")
    xb = pcf.PcfTensors.from_numpy(B, "cuda")
    specs = ["l1", "l2", ("lp", 3.0)]
    host = pcf.pcf_cross_to_host(xa, xb, specs, precision="f32c", block_rows=1024,
                                 out_dtype=torch.float32)
    rng = np.random.default_rng(19)
    ii = rng.integers(0, rows.n, 1000)
    jj = rng.integers(0, B.n, 1000)
    for (name, p), h in zip((("l1", 1.0), ("l2", 2.0), ("lp", 3.0)), host):
        got = h.numpy()[ii, jj].astype(np.float64)
        _check_entries(rows, got, ii, jj, name, p, TOL["f32c"], b=B)
