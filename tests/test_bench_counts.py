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


def test_launch_resolution():
    """--gpus N: one process runs alone only for N = 1; N > 1 outside a
    launcher spawns N ranks, and under a launcher WORLD_SIZE must equal N."""
    assert bench.resolve_launch(1, {}, 1) == ("run", 1)
    assert bench.resolve_launch(2, {}, 8) == ("spawn", 2)
    assert bench.resolve_launch(4, {}, 2)[0] == "error"          # not enough GPUs
    env = {"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0"}
    assert bench.resolve_launch(2, env, 2) == ("run", 2)
    assert bench.resolve_launch(4, env, 8)[0] == "error"         # launcher disagrees
    assert bench.resolve_launch(1, env, 8)[0] == "error"
    assert bench.resolve_launch(0, {}, 8)[0] == "error"


def test_spawn_command_is_a_torchrun_of_this_script():
    cmd = bench.spawn_command(4, ["--gpus", "4", "--steps", "3"], 29555)
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert "--nproc-per-node=4" in cmd
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[cmd.index("--master-port") + 1] == "29555"
    i = next(k for k, c in enumerate(cmd) if c.endswith("bench.py"))
    assert cmd[i + 1:] == ["--gpus", "4", "--steps", "3"]


def test_split_value_is_set_by_the_slowest_rank():
    assert bench.split_value(1000, [2.0, 4.0, 3.0]) == 1000 / 4e-3


def test_matrix_errors_measure():
    """Distances relative to the entry (a nonzero where the oracle has an exact
    0 is an infinite error); Gram against sqrt(G*_ii G*_jj)."""
    want = {"l1": np.array([[0.0, 2.0], [2.0, 0.0]]), "l2": np.array([[0.0, 4.0], [4.0, 0.0]]),
            "gram": np.array([[4.0, 1.0], [1.0, 9.0]])}
    got = {"l1": np.array([[0.0, 2.2], [2.0, 0.0]]), "l2": want["l2"].copy(),
           "gram": np.array([[4.0, 1.6], [1.0, 9.0]])}
    e = bench.matrix_errors(got, want, np.array([4.0, 9.0]), 0)
    assert abs(e["l1"] - 0.1) < 1e-12 and e["l2"] == 0.0 and abs(e["gram"] - 0.1) < 1e-12
    got["l2"][0, 0] = 1e-9
    assert bench.matrix_errors(got, want, np.array([4.0, 9.0]), 0)["l2"] == float("inf")


def test_one_gpu_workloads_refuse_several_ranks():
    """Under a launcher with two ranks, a workload that runs on one GPU only
    (every secondary workload but the gradient) stops with an error line and
    exit code 2 before any device work; the gradient workload is the one
    secondary workload that splits over ranks."""
    import json
    import subprocess
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0",
               MASTER_ADDR="127.0.0.1", MASTER_PORT="29613")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                        "--workload", "uniform_small"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 2, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert "runs on one GPU" in line["error"]
    assert bench.MULTI_RANK_WORKLOADS == ("gradient",)
