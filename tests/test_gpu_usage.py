"""The documented Python usage runs and agrees with the oracle (needs a GPU)."""
import numpy as np
import pytest

import oracle
from paper_2404_07183_gb300 import synth

from conftest import gpu_available

pytestmark = pytest.mark.gpu


def test_documented_usage():
    if not gpu_available():
        pytest.skip("no CUDA device")
    import torch

    import paper_2404_07183_gb300 as pcf
    pcf.build.build()
    s = synth.stable_rank(n_pcfs=400)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    l1, l2, gram = pcf.pcf_pairwise(x, ["l1", "l2", "gram"], precision="f32c")
    d35 = pcf.pdist(x, p=3.5)
    G = pcf.l2_kernel(x)
    block = pcf.pcf_cross(x, x, 0, 128, [("lp", 3.0)])[0]
    gv, gt = pcf.pcf_pairwise_backward(x, ("l2", False),
                                       torch.randn(400, 400, device="cuda", dtype=torch.float64))
    w = pcf.pcf_pairwise(x, ["l1"], window=(1.0, 30.0, 0.1))[0]
    norms = pcf.pcf_segment_integrals(x, "lp", 2.0, apply_root=True)
    m = pcf.mean(x, group_size=100)
    sd = pcf.std(x, group_size=100)
    dev = pcf.pcf_combine(x, pcf.mean(x), "sub")
    torch.cuda.synchronize()

    want = oracle.matrix(s, metric="l1")
    assert np.max(np.abs(l1.cpu().numpy() - want) / np.where(want == 0, 1, want)) < 1e-5
    want = oracle.matrix(s, metric="lp", p=3.5)
    assert np.max(np.abs(d35.cpu().numpy() - want) / np.where(want == 0, 1, want)) < 1e-12
    np.testing.assert_allclose(np.diag(G.cpu().numpy()), norms.cpu().numpy() ** 2, rtol=1e-12)
    assert block.shape == (128, 400) and gv.shape == (s.nnz,) and gt.shape == (s.nnz,)
    i, j = 3, 7
    want = oracle.integral_ab(*s.pcf(i), *s.pcf(j), "l1", 1.0, 1.0, 30.0, 0.1)
    assert abs(float(w[i, j]) - want) <= 1e-5 * want
    for got, red, g in ((m, "mean", 100), (sd, "std", 100)):
        off, t, v = oracle.reduce(s, g, red)
        np.testing.assert_array_equal(got.offsets.cpu().numpy(), off)
        np.testing.assert_array_equal(got.values.cpu().numpy(), v)
    assert dev.n == s.n
    np.testing.assert_array_equal(l2.cpu().numpy(), l2.cpu().numpy().T)
    assert gram.dtype == torch.float32
