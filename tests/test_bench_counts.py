"""The benchmark's exact merge-step counters agree with the oracle's count of
rectangles |T_f u T_g| (host logic, no GPU)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2404_07183_gb300 import synth  # noqa: E402


def test_pairwise_step_count_matches_oracle():
    for s in (synth.dyadic(30, seed=3, max_len=20), synth.lognormal(150, seed=5),
              synth.stable_rank(40)):
        w, d = bench.exact_walk_steps(s)
        assert w + d == oracle.total_merge_steps(s)
