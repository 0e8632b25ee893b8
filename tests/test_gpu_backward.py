"""Adjoint kernel vs the oracle adjoint (needs a GPU).

Error measure per gradient array: max |g - g*| / max |g*| <= 1e-12 for random
inputs; bit-exact on dyadic inputs with shared breakpoints (every term is an
exact small dyadic number, so the order of the float64 atomics cannot change
the sums).
"""
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


def _spec(metric, p, root):
    if metric == "lp":
        return ("lp", p, root)
    return (metric, root)


def _rel(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


CASES = [("l2", 2.0, False), ("l1", 1.0, False), ("gram", 1.0, False), ("lp", 3.0, False),
         ("lp", 2.5, True), ("l2", 2.0, True), ("l1", 1.0, True)]


@pytest.mark.parametrize("metric,p,root", CASES)
def test_backward_vs_oracle(pcf, metric, p, root):
    import torch
    s = synth.random_set(70, seed=51, min_len=2, max_len=40)
    G = np.random.default_rng(3).standard_normal((s.n, s.n))
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    Gt = torch.from_numpy(G).cuda()
    F = None
    if root:
        F = pcf.pcf_pairwise(x, [_spec(metric, p, True)], precision="f64",
                             out_dtype=torch.float64)[0]
    gv, gt = pcf.pcf_pairwise_backward(x, _spec(metric, p, root), Gt, fwd_out=F)
    ov, ot = oracle.backward(s, G, metric=metric, p=p, apply_root=root)
    assert _rel(gv.cpu().numpy(), ov) <= 1e-12
    assert _rel(gt.cpu().numpy(), ot) <= 1e-12


@pytest.mark.parametrize("metric", ["l2", "gram", "l1"])
def test_backward_dyadic_bitwise(pcf, metric):
    import torch
    s = synth.dyadic(90, seed=52, max_len=30, min_len=1, max_gap=3, max_abs_value=5)
    rng = np.random.default_rng(4)
    G = rng.integers(-8, 9, size=(s.n, s.n)) / 8.0
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    gv, gt = pcf.pcf_pairwise_backward(x, (metric, False), torch.from_numpy(G).cuda())
    ov, ot = oracle.backward(s, G, metric=metric, p=2.0)
    np.testing.assert_array_equal(gv.cpu().numpy(), ov)
    np.testing.assert_array_equal(gt.cpu().numpy(), ot)


def test_autograd_function(pcf):
    import torch
    s, G = synth.gradient(200)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    values = x.values.clone().requires_grad_(True)
    times = x.times.clone().requires_grad_(True)
    F = pcf.PairwiseFn.apply(values, times, x.offsets, ("l2", False), "f64")
    loss = (torch.from_numpy(G).cuda() * F).sum()
    loss.backward()
    ov, ot = oracle.backward(s, G, metric="l2", p=2.0)
    assert _rel(values.grad.cpu().numpy(), ov) <= 1e-12
    assert _rel(times.grad.cpu().numpy(), ot) <= 1e-12
    want = float(np.sum(G * oracle.matrix(s, metric="l2", apply_root=False)))
    assert abs(loss.item() - want) <= 1e-12 * abs(want)


def test_gradient_workload_full_size_sampled(pcf):
    """N = 4,096 PCFs, loss = sum(G * D2^2): gradients of a sample of PCFs
    against the oracle restricted to the pairs touching them."""
    import torch
    s, G = synth.gradient()
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    gv, gt = pcf.pcf_pairwise_backward(x, ("l2", False), torch.from_numpy(G).cuda())
    gv, gt = gv.cpu().numpy(), gt.cpu().numpy()
    rng = np.random.default_rng(9)
    for i in rng.choice(s.n, 4, replace=False):
        # the gradient of PCF i only depends on the pairs (i, j): build a
        # 2-row problem per partner and sum the oracle's gradients for i
        ti, vi = s.pcf(i)
        acc_v = np.zeros(ti.size)
        acc_t = np.zeros(ti.size)
        for j in range(s.n):
            if j == i:
                continue
            tj, vj = s.pcf(j)
            sub = synth.PcfSet(np.array([0, ti.size, ti.size + tj.size]),
                               np.concatenate([ti, tj]), np.concatenate([vi, vj]))
            g2 = np.array([[0.0, G[i, j]], [G[j, i], 0.0]])
            ov, ot = oracle.backward(sub, g2, metric="l2", p=2.0)
            acc_v += ov[:ti.size]
            acc_t += ot[:ti.size]
        a, b = int(s.offsets[i]), int(s.offsets[i + 1])
        assert _rel(gv[a:b], acc_v) <= 1e-12
        assert _rel(gt[a:b], acc_t) <= 1e-12


@pytest.mark.parametrize("world", [2, 3])
def test_backward_shards_sum_to_the_gradient(pcf, world):
    """One matrix's gradient split over `world` GPUs (run here one after the
    other): the shards' partial gradients sum to the unsharded one."""
    import torch
    s = synth.random_set(150, seed=131, min_len=2, max_len=60)
    x = pcf.PcfTensors.from_numpy(s, "cuda")
    G = torch.randn(s.n, s.n, device="cuda", dtype=torch.float64)
    for spec in (("l2", False), "gram", ("lp", 2.5, True)):
        fwd = None
        if spec == ("lp", 2.5, True):
            fwd = pcf.pcf_pairwise(x, [spec], precision="f64", out_dtype=torch.float64)[0]
        gv, gt = pcf.pcf_pairwise_backward(x, spec, G, fwd_out=fwd)
        sv = torch.zeros_like(gv)
        st = torch.zeros_like(gt)
        for r in range(world):
            pv, pt = pcf.pcf_pairwise_backward(x, spec, G, fwd_out=fwd, shard=(r, world))
            sv += pv
            st += pt
        assert _rel(sv.cpu().numpy(), gv.cpu().numpy()) < 1e-12, spec
        assert _rel(st.cpu().numpy(), gt.cpu().numpy()) < 1e-12, spec
