"""pcf_pairwise_noalloc: the entry point for callers that cannot allocate
device memory (their scratch is a fixed device array inside the library).

Called through the C ABI and compared with pcf_pairwise, which uses a caller
workspace, on two calls in a row (the second call must not see anything left
over from the first).  Both paths run the same kernels in the same order on
the same inputs, so their matrices must agree bit for bit; a tolerance could
hide state left in the shared array.  Collected last so that a failure here
does not stop a -x run before the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2404_07183_gb300 import abi, synth

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2404_07183_gb300 import build
    build.build()
    return abi.load()


def _noalloc(lib, x, metrics, precision, outs):
    import torch
    import paper_2404_07183_gb300 as P
    from paper_2404_07183_gb300.api import _requests, _prec
    req = _requests(metrics, outs)
    cx = x.csr()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.pcf_pairwise_noalloc(ctypes.byref(cx), req, len(metrics), _prec(precision),
                                  abi.PCF_OUT_FULL, abi.PCF_F64, stream)
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("precision", ["f64", "f32c"])
def test_noalloc_matches_workspace_path_twice(lib, precision):
    import torch
    import paper_2404_07183_gb300 as P
    metrics = ["l1", "l2", "gram"]
    a = synth.uniform_small(n_pcfs=300, seed=71)
    b = synth.uniform_small(n_pcfs=257, seed=72)
    for s in (a, b):   # two calls in a row, different sizes: no leftovers
        x = P.PcfTensors.from_numpy(s, "cuda")
        want = P.pcf_pairwise(x, metrics, precision=precision, out_dtype=torch.float64)
        outs = [torch.full((s.n, s.n), np.nan, dtype=torch.float64, device="cuda")
                for _ in metrics]
        assert _noalloc(lib, x, metrics, precision, outs) == abi.PCF_OK
        for o, w in zip(outs, want):
            np.testing.assert_array_equal(o.cpu().numpy(), w.cpu().numpy())


def test_noalloc_invalid_input_then_valid_call(lib):
    """A call on invalid PCF data (times not increasing) returns PCF_OK, as
    device-side data errors are not reported by this entry point, and leaves
    the device usable; the next valid call clears the error word it left in
    the shared array and matches the workspace path exactly."""
    import torch
    import paper_2404_07183_gb300 as P
    metrics = ["l1", "gram"]
    s = synth.uniform_small(n_pcfs=120, seed=73)
    t = s.times.copy()
    k = int(s.offsets[5]) + 2
    t[k] = t[k - 1]                     # a repeated breakpoint
    bad = P.PcfTensors.from_numpy(synth.PcfSet(s.offsets, t, s.values), "cuda")
    outs = [torch.zeros((s.n, s.n), dtype=torch.float64, device="cuda") for _ in metrics]
    assert _noalloc(lib, bad, metrics, "f64", outs) == abi.PCF_OK
    good = P.PcfTensors.from_numpy(s, "cuda")
    want = P.pcf_pairwise(good, metrics, precision="f64", out_dtype=torch.float64)
    outs = [torch.full((s.n, s.n), np.nan, dtype=torch.float64, device="cuda") for _ in metrics]
    assert _noalloc(lib, good, metrics, "f64", outs) == abi.PCF_OK
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w.cpu().numpy())


def test_noalloc_rejects_inputs_beyond_the_scratch(lib):
    c = abi.PcfCsr()
    c.n, c.nnz, c.dtype = 100000, abi.PCF_NOALLOC_SCRATCH_BYTES, abi.PCF_F64
    c.offsets = c.times = c.values = 0x1000
    req = (abi.PcfIntegral * 1)()
    req[0].metric, req[0].p, req[0].out = abi.PCF_L1, 1.0, 0x2000
    rc = lib.pcf_pairwise_noalloc(ctypes.byref(c), req, 1, abi.PCF_PREC_F64,
                                  abi.PCF_OUT_FULL, abi.PCF_F64, ctypes.c_void_p(0))
    assert rc == abi.PCF_ENOWS
