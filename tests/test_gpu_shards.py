"""Logical shards on one GPU: the shards of one matrix, computed one after
another, add up to the unsharded result bit for bit (needs a GPU)."""
import numpy as np
import pytest

from paper_2404_07183_gb300 import shard, synth

from conftest import gpu_available

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sched", ["tile1024", "tile512x2", "mergepath"])
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
