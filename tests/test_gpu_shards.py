"""Logical shards on one GPU: the shards of one matrix, computed one after
another, add up to the unsharded result bit for bit (needs a GPU)."""
import numpy as np
import pytest

from paper_2404_07183_gb300 import shard, synth

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sched", ["tile1024", "tile512x2", "tile512x3", "mergepath"])
@pytest.mark.parametrize("world", [2, 3])
def test_shards_sum_to_the_whole(sched, world):
    if not gpu_available():
        pytest.skip("no CUDA device")
    import torch
    import paper_2404_07183_gb300 as P
    s = synth.random_set(150, seed=95, min_len=1, max_len=80)
    x = P.PcfTensors.from_numpy(s, "cuda")
    whole = P.pcf_pairwise(x, ["l1", "gram"], precision="f64", out_dtype=torch.float64,
                           schedule=sched)
    total = [torch.zeros_like(w) for w in whole]
    for r in range(world):
        part = shard.pairwise_shard(x, ["l1", "gram"], r, world, precision="f64",
                                    out_dtype=torch.float64, schedule=sched)
        for t, p_ in zip(total, part):
            t += p_
    for t, w in zip(total, whole):
        np.testing.assert_array_equal(t.cpu().numpy(), w.cpu().numpy())


@pytest.mark.parametrize("n_short,n_long,sched", [(60, 40, "tile1024"), (500, 140, "tile1024"),
                                                  (500, 140, "tile512x2")])
def test_host_mirror_matches_device_ownership(n_short, n_long, sched):
    """The host mirror of the sort (length, then time scale for PCFs longer
    than 256 points) and of the tile order (bands of column blocks; 640 PCFs
    make 20 blocks, two bands) names exactly the entries the device writes
    for a shard."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    import torch
    import paper_2404_07183_gb300 as P
    rng = np.random.default_rng(7)
    lens = np.concatenate([rng.integers(2, 60, n_short), rng.integers(257, 700, n_long)])
    scales = np.exp(rng.normal(0, 1.5, lens.size))
    s = synth.from_lengths(lens, lambda r, m: r.exponential(1.0, m),
                           lambda r, o: r.standard_normal(o[-1]) + 3.0, rng, np.float64, "scaled")
    t = s.times.copy()
    for i in range(s.n):
        a, b = int(s.offsets[i]), int(s.offsets[i + 1])
        t[a:b] *= scales[i]
    s = synth.PcfSet(s.offsets, t, s.values)
    x = P.PcfTensors.from_numpy(s, "cuda")
    last = s.times[s.offsets[1:] - 1]
    for r in range(3):
        part = shard.pairwise_shard(x, ["gram"], r, 3, precision="f64",
                                    out_dtype=torch.float64, schedule=sched)[0].cpu().numpy()
        got = {(i, j) for i, j in zip(*np.nonzero(part)) if i <= j}
        want = shard.shard_pairs(s.lengths(), r, 3, last_times=last)
        assert got == want
