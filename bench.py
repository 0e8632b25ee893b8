"""Benchmark of the pairwise PCF integral-matrix path on GB300.

Default workload: N = 20,000 stable-rank-like PCFs (n ~ U{50..500}, Exp(0.1)
gaps, non-increasing integer values 200 -> 0), L1 distance + L2 distance + L2
Gram matrices in one fused walk per pair, float32-compensated walk (headline)
and the float64 walk side by side; outputs are full N x N float32 matrices.

One step = the whole hot path on device-resident input: validate + length
sort + pack (pcf_prepare) and the persistent tile walk (pcf_pairwise with
PCF_PAIRWISE_PREPARED).  L2 is flushed (256 MiB write) before every timed
step, outside the per-step CUDA-event brackets.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(threaded float64 walk) on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2404_07183_gb300 import synth  # noqa: E402

METRICS = ["l1", "l2", "gram"]
# the headline metric and workload, shared by both arms of the benchmark
HEADLINE_METRIC = ("pair-integrals/s and merge-steps/s at 1 GB300 (FP32-comp vs FP64), "
                   "% issue roofline")
HEADLINE_WORKLOAD = "stable_rank N=20000 n~U{50..500} Exp(0.1) gaps, L1+L2+Gram fused"
# Algorithmic operations per merge step (frozen tally, see the design notes):
# common part 5 (compare, select rectangle end, dt, fetch, advance) + d = a-b 1
# L1 |d|*dt fma 1, L2 d*d + fma 2, Gram a*b + fma 2; compensated (Kahan): each
# accumulate is the fma that subtracts the compensation plus 3 additions.
TALLY = {"f32c": 5 + 1 + (1 + 3) + (2 + 3) + (2 + 3), "f32": 5 + 1 + 1 + 2 + 2,
         "f64": 5 + 1 + 1 + 2 + 2,
         # block-compensated: plain FMA terms + one 4-op Kahan add per metric per 16 steps
         "f32b": 5 + 1 + 1 + 2 + 2 + 3 * 4 / 16}
# float64 input walked in float32 with exact comparisons (order keys): the
# rectangle end is selected as hi and lo (one more select) and its width is
# (hi_n - hi_c) + (lo_n - lo_c) (two more operations): common part 8 instead of 5
KEYED_EXTRA = 3
# float64 times rounded to float32 when packed (opt-in): the round-1 form
for _p in ("f32c", "f32b", "f32"):
    TALLY[_p + "_round"] = TALLY[_p]


def tally(prec, input_f64=True):
    """Operations per merge step of the walk a precision name runs on this input."""
    keyed = input_f64 and prec in ("f32c", "f32b", "f32")
    return TALLY[prec] + (KEYED_EXTRA if keyed else 0)
FP64_OPS_PER_STEP = 1 + 1 + 1 + 2 + 2   # dt, d, L1 fma, L2 mul+fma, Gram mul+fma

# DRAM bytes (read + write) per launch of the benchmark's compensated walk,
# from one ncu capture (profiles/walk_f32ck_dram_traffic_stable_rank_n20000.md),
# valid only while the walk's source is the one that was measured.
TRAFFIC_RECORD = {"source_sha256_16": "cc8a5afd078a05bc+cbd8c1c574e4db57",
                  "by_schedule_layout": {("tile512x2", "full"): 1206109440 + 4928763392}}


def walk_source_id():
    import hashlib
    parts = []
    for f in ("walk.cuh", "internal.cuh"):
        with open(os.path.join(ROOT, "paper_2404_07183_gb300", "csrc", f), "rb") as fh:
            parts.append(hashlib.sha256(fh.read()).hexdigest()[:16])
    return "+".join(parts)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_launches(prec, layout="full", input_f64=True):
    """Kernels one timed step launches: pcf_prepare (header, validation,
    length sort, pack; for float64 input in a float32 walk the key sort: key
    count, 8 passes of histogram + two row scans + scatter, distinct-key
    count, its scan and the rank write), pcf_pairwise (tile counter, walk;
    FULL layout: inverse permutation and the column pass)."""
    keyed = input_f64 and prec in ("f32c", "f32b", "f32")
    n = 4 + (1 + 8 * 4 + 3 if keyed else 0) + 2
    return n + (2 if layout == "full" else 0)


def resolve_launch(gpus, env, device_count):
    """What to do with ``--gpus N`` in this process: ("run", world) when the
    process is one of the N ranks (WORLD_SIZE == N under torchrun, or N == 1),
    ("spawn", N) when N > 1 ranks must be started (no torchrun around us), or
    ("error", message) when the launch cannot give N ranks on this node."""
    world = int(env.get("WORLD_SIZE", "1"))
    under_launcher = "RANK" in env and "WORLD_SIZE" in env
    if gpus < 1:
        return "error", f"--gpus {gpus}: need at least one GPU"
    if under_launcher:
        if world != gpus:
            return "error", f"--gpus {gpus} but the launcher started WORLD_SIZE={world} ranks"
        return "run", world
    if gpus == 1:
        return "run", 1
    if device_count < gpus:
        return "error", f"--gpus {gpus} but this node has {device_count} GPU(s)"
    return "spawn", gpus


def spawn_command(gpus, argv, port):
    """torchrun command that starts ``gpus`` ranks of this script (one per GPU)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            f"--nproc-per-node={gpus}", "--master-addr", "127.0.0.1", "--master-port", str(port),
            os.path.abspath(__file__)] + list(argv)


def split_value(pairs, step_ms_per_rank):
    """Whole-matrix throughput of one matrix split over ranks: all of its
    pairs over the slowest rank's step time (strong scaling)."""
    return pairs / (max(step_ms_per_rank) * 1e-3)


def exact_walk_steps(s):
    """sum over pairs i < j of |T_i u T_j| plus sum_i |T_i| (Gram diagonal):
    |T_i u T_j| = n_i + n_j - |T_i n T_j|; t = 0 is shared by every pair and a
    positive time shared by c PCFs is shared by c(c-1)/2 pairs."""
    N, nnz = s.n, s.nnz
    t = np.asarray(s.times, dtype=np.float64)
    pos = t[t > 0]
    _, counts = np.unique(pos, return_counts=True)
    shared = int(np.sum(counts * (counts - 1) // 2))
    pairs = (N - 1) * nnz - N * (N - 1) // 2 - shared
    return int(pairs), int(nnz)


def workload(rank=0, n=None):
    if n:
        return synth.stable_rank(n_pcfs=n, seed=1002 + rank)
    return synth.stable_rank(seed=1002 + rank)


def start_clock_sampler(path):
    try:
        fh = open(path, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=fh, stderr=subprocess.DEVNULL)
        return p, fh
    except Exception:
        return None, None


def stop_clock_sampler(p, fh, path, gpu_index):
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    fh.close()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or f[0] != str(gpu_index):
            continue
        try:
            sm.append(float(f[1]))
            mx = max(mx, float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def pipe_peaks():
    """FP64 and FP32 FMA lane rates per SM per clock (own microbenchmark)."""
    from paper_2404_07183_gb300 import build
    lib = ctypes.CDLL(build.build_peaks())
    lib.pcf_peak_fma.restype = ctypes.c_int
    lib.pcf_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for name, f64, iters in (("fp64", 1, 2000), ("fp32", 0, 50000)):
        clk, rate = ctypes.c_double(), ctypes.c_double()
        rc = lib.pcf_peak_fma(f64, sms, iters, ctypes.byref(clk), ctypes.byref(rate))
        out[name] = {"lane_ops_per_clk_per_sm": clk.value, "lane_ops_per_s": rate.value, "rc": rc}
    out["sms"] = sms
    return out


# --------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    s = workload()
    cores = len(os.sched_getaffinity(0))
    rows_per_step = args.ref_rows
    steps_rows = []
    times = []
    total_pairs = 0
    rng = np.random.default_rng(0)
    for k in range(args.warmup + args.steps):
        r0 = int(rng.integers(0, s.n - rows_per_step))
        t0 = time.perf_counter()
        for m in METRICS:
            oracle.matrix(s, metric=m, rows=(r0, r0 + rows_per_step), nthreads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            steps_rows.append(r0)
            total_pairs += 3 * rows_per_step * s.n
    elapsed = sum(times)
    value = total_pairs / elapsed
    line = {
        "impl": "reference", "metric": HEADLINE_METRIC,
        "value": value, "unit": "pair-integrals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": HEADLINE_WORKLOAD, "N": s.n, "nnz": s.nnz, "metrics": METRICS,
                   "precision": "f64 (CPU oracle walk)",
                   "sample": f"{rows_per_step} consecutive rows x {s.n} columns per step"},
        "cpu_baseline": {"value": value, "unit": "pair-integrals/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{rows_per_step} rows x {s.n} cols x 3 metrics per step"},
        "e2e": {"value": value, "unit": "pair-integrals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SAMPLE_ROW0 = 1000        # first row of the oracle's timed sample (and of the error check)


def cpu_baseline(s, seconds_target=15.0, max_rows=None):
    """The oracle timed on a bounded row sample of the workload (all host
    cores).  Returns (record, oracle rows per metric, Gram diagonal): the
    sampled rows are also the reference of the per-matrix error check."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    r0 = SAMPLE_ROW0
    oracle.matrix(s, metric="l1", rows=(r0, r0 + 2), nthreads=cores)   # load + thread start
    rows = 16
    t0 = time.perf_counter()
    oracle.matrix(s, metric="l1", rows=(r0, r0 + rows), nthreads=cores)
    dt = time.perf_counter() - t0
    # three metrics of about seconds_target / 3 each, on the calibrated rows
    rows = int(max(16, min(s.n - r0, rows * (seconds_target / 3.0) / max(dt, 1e-3))))
    if max_rows:
        rows = min(rows, max_rows)
    t0 = time.perf_counter()
    want = {m: oracle.matrix(s, metric=m, rows=(r0, r0 + rows), nthreads=cores) for m in METRICS}
    dt = time.perf_counter() - t0
    diag = np.array([oracle.segment_sq(*s.pcf(i)) for i in range(s.n)])
    rec = {"value": 3 * rows * s.n / dt, "unit": "pair-integrals/s", "cores": cores,
           "kind": "oracle", "seconds": dt,
           "sample": f"rows {r0}..{r0 + rows} x all {s.n} columns, L1+L2+Gram, "
                     "float64 oracle walk, one thread per core"}
    return rec, want, diag


def matrix_errors(got, want, diag, r0):
    """Per-matrix error of GPU rows against the oracle's rows: distances
    max |x - x*| / |x*| (x* = 0 only on the diagonal, which must be exactly 0);
    Gram max |x - x*| / sqrt(G*_ii G*_jj)."""
    out = {}
    for m in METRICS:
        g = np.asarray(got[m], dtype=np.float64)
        w = np.asarray(want[m], dtype=np.float64)
        rows = g.shape[0]
        if m == "gram":
            d = np.sqrt(np.abs(diag))
            scale = np.outer(d[r0:r0 + rows], d)
            scale = np.where(scale > 0, scale, 1.0)
            out[m] = float(np.max(np.abs(g - w) / scale))
        else:
            zero = w == 0
            if np.any(g[zero] != 0):
                out[m] = float("inf")
                continue
            out[m] = float(np.max(np.abs(g - w)[~zero] / np.abs(w[~zero])))
    return out


def _broadcast_set(s, local, world, rank):
    """The collection on every rank: rank 0's arrays broadcast over NCCL (the
    other ranks pass s = None)."""
    import torch
    import torch.distributed as dist
    import paper_2404_07183_gb300 as P
    dev = f"cuda:{local}"
    if rank == 0:
        x = P.PcfTensors.from_numpy(s, dev)
        sizes = torch.tensor([x.n, x.nnz, 1 if x.times.dtype == torch.float64 else 0],
                             dtype=torch.int64, device=dev)
    else:
        sizes = torch.zeros(3, dtype=torch.int64, device=dev)
    dist.broadcast(sizes, 0)
    n, nnz, f64 = (int(v) for v in sizes.tolist())
    if rank != 0:
        dt = torch.float64 if f64 else torch.float32
        x = P.PcfTensors(torch.empty(n + 1, dtype=torch.int64, device=dev),
                         torch.empty(nnz, dtype=dt, device=dev),
                         torch.empty(nnz, dtype=dt, device=dev))
    for t in (x.offsets, x.times, x.values):
        dist.broadcast(t, 0)
    return x


def run_ours(args):
    import torch
    import paper_2404_07183_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    split = world > 1 and not args.replicas
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.build.build()

    # split: one matrix over all ranks, broadcast from rank 0 (strong scaling);
    # replicas: an independent batch per rank (weak scaling)
    s = workload(0 if split else rank, args.n) if (rank == 0 or not split) else None
    if split:
        x = _broadcast_set(s, local, world, rank)
    else:
        x = P.PcfTensors.from_numpy(s, f"cuda:{local}")
    N = x.n
    shard = (rank, world) if split else None
    walk_steps, diag_steps = exact_walk_steps(s) if s is not None else (0, 0)
    pairs = 2 * (N * (N - 1) // 2) + N * (N + 1) // 2      # distances i<j, Gram i<=j
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    check_rows = (SAMPLE_ROW0, min(N, SAMPLE_ROW0 + args.check_rows))
    check = (world == 1 and not args.no_cpu and N > SAMPLE_ROW0)

    def make_outs():
        return [torch.empty((N, N), dtype=torch.float32, device=f"cuda:{local}") for _ in METRICS]

    results = {}
    tuned = {}
    samples = {}
    forms = [args.precision]
    if not args.no_fp64:
        forms += [f for f in ("f32b", "f64", "f32c_round") if f != args.precision]
    for prec in forms:
        if args.schedule:
            sched = args.schedule
        else:
            from paper_2404_07183_gb300 import autotune
            sched, timings = autotune.tune_pairwise(x, METRICS, prec, repeats=1)
            tuned[prec] = {"schedule": sched, "timings_ms": timings}
            if split:
                # every rank walks its shard with rank 0's choice
                obj = [sched]
                torch.distributed.broadcast_object_list(obj, 0)
                sched = obj[0]
        outs = make_outs()
        ws = torch.empty(P.pcf_workspace_size(x, None, prec), dtype=torch.uint8,
                         device=f"cuda:{local}")

        def step():
            P.pcf_prepare(x, prec, workspace=ws)
            e_mid = torch.cuda.Event(enable_timing=True)
            e_mid.record(stream)
            P.pcf_pairwise(x, METRICS, precision=prec, out=outs, workspace=ws, prepared=True,
                           check=False, schedule=sched, layout=args.layout, shard=shard)
            return e_mid

        steps = args.steps if prec == args.precision else max(1, min(args.steps, 2))
        warm = args.warmup
        for _ in range(warm):
            step()
        P.pcf_check(ws)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        sampler, sfh = (None, None)
        clk_path = os.path.join(tempfile.gettempdir(), f"pcf_bench_clocks_{prec}_r{rank}.csv")
        if prec == args.precision:
            os.makedirs(os.path.dirname(clk_path), exist_ok=True)
            sampler, sfh = start_clock_sampler(clk_path)
        t_wall = time.perf_counter()
        evs = []
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e1 = step()
            e2.record(stream)
            evs.append((e0, e1, e2))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t_wall = time.perf_counter() - t_wall
        clocks = stop_clock_sampler(sampler, sfh, clk_path, local) if sampler else None
        P.pcf_check(ws)
        step_ms = [a.elapsed_time(c) for a, b, c in evs]
        walk_ms = [b.elapsed_time(c) for a, b, c in evs]
        tot = sum(step_ms)
        if world > 1:
            t = torch.tensor([tot], device=f"cuda:{local}", dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            tot = float(t.item())
        results[prec] = {"schedule": sched, "ms_per_step": tot / steps,
                         "walk_ms": float(np.mean(walk_ms)),
                         "prepare_ms": float(np.mean([a.elapsed_time(b) for a, b, c in evs])),
                         "steps": steps, "wall_s": t_wall, "clocks": clocks}
        if check and args.layout == "full":
            r0, r1 = check_rows
            samples[prec] = {m: o[r0:r1].double().cpu().numpy() for m, o in zip(METRICS, outs)}
        del outs, ws

    # same walk writing the matrices in the library's sort order (tiles land in
    # contiguous blocks instead of being scattered by the permutation)
    sorted_walk = None
    if not args.no_fp64 and args.layout == "full" and world == 1:
        prec = args.precision
        outs_s = make_outs()
        ws_s = torch.empty(P.pcf_workspace_size(x, None, prec), dtype=torch.uint8,
                           device=f"cuda:{local}")
        P.pcf_prepare(x, prec, workspace=ws_s)

        def sstep():
            P.pcf_pairwise(x, METRICS, precision=prec, out=outs_s, workspace=ws_s, prepared=True,
                           check=False, schedule=results[prec]["schedule"], layout="sorted")
        sms_ = _timed(sstep, 2, 1, flush, stream)
        P.pcf_check(ws_s)
        sorted_walk = float(np.mean(sms_))
        del outs_s, ws_s

    if args.no_e2e:
        if rank == 0:
            print(json.dumps({"results": results, "N": N, "walk_steps": walk_steps}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    # end-to-end through the public API with host buffers (pinned), every step:
    # H2D of the CSR, the whole path, the matrices read back to the host.  One
    # GPU: the three matrices streamed to the host band by band while the walk
    # runs (pcf_pairwise_to_host).  A split matrix: each rank walks its shard
    # and reads back its matrices (entries outside its shard are not its own).
    prec = args.precision
    host_in = [torch.from_numpy(np.ascontiguousarray(a.cpu().numpy())).pin_memory()
               for a in (x.offsets, x.times, x.values)]
    host_out = [torch.empty((N, N), dtype=torch.float32).pin_memory() for _ in METRICS]
    dev_in = [torch.empty_like(h, device=f"cuda:{local}") for h in host_in]
    outs = make_outs()
    ws = torch.empty(P.pcf_workspace_size(x, None, prec), dtype=torch.uint8, device=f"cuda:{local}")
    h2d = sum(h.numel() * h.element_size() for h in host_in)
    d2h = sum(h.numel() * h.element_size() for h in host_out)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    phases = []
    copy_stream = torch.cuda.Stream(f"cuda:{local}")

    def e2e_step():
        ev[0].record()
        for d, h in zip(dev_in, host_in):
            d.copy_(h, non_blocking=True)
        ev[1].record()
        xd = P.PcfTensors(*dev_in)
        ev[2].record()
        if split:
            P.pcf_pairwise(xd, METRICS, precision=prec, out=outs, workspace=ws, check=False,
                           schedule=results[prec]["schedule"], shard=shard)
            for h, o in zip(host_out, outs):
                h.copy_(o, non_blocking=True)
        else:
            P.pcf_pairwise_to_host(xd, METRICS, precision=prec, out=outs, host_out=host_out,
                                   workspace=ws, check=False, schedule=results[prec]["schedule"],
                                   copy_stream=copy_stream)
        ev[3].record()

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
        torch.cuda.synchronize()
        phases.append([ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])])
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    P.pcf_check(ws)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peaks = measured_peaks()
    pp = pipe_peaks()
    sms = pp["sms"]
    fmax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    head = results[prec]
    units = 1 if split else world           # matrices computed per step by the whole job
    value = units * pairs / (head["ms_per_step"] * 1e-3)
    walk_rate = walk_steps / (head["walk_ms"] * 1e-3) if not split else None
    issue_peak = sms * 128 * fmax / tally(prec)
    line = {
        "metric": HEADLINE_METRIC,
        "value": value, "unit": "pair-integrals/s", "n_gpus": world, "steps": head["steps"],
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "strong" if split else "weak", "vs_baseline": None,
        "dtype": "f32 (compensated)", "data": "synthetic",
        "config": {"workload": HEADLINE_WORKLOAD,
                   "N": N, "nnz": x.nnz, "metrics": METRICS, "precision": prec,
                   "comparisons": "exact in float64 (order keys ranked from the float64 times)"
                                  if "round" not in prec else "on float32-rounded times",
                   "layout": "full N x N", "out_dtype": "f32",
                   "pair_integrals_per_step": units * pairs,
                   "merge_steps_per_step": units * (walk_steps + diag_steps),
                   "l2": "flushed by a 256 MiB write before each timed step (outside the timing)",
                   "parallelism": (f"one matrix split over {world} GPUs (strided 32x32 tile "
                                   "shards, input broadcast from rank 0)" if split
                                   else f"{world} independent replicas (one per GPU)"),
                   "schedule": head["schedule"], "autotune": tuned or None},
        "merge_steps_per_s": units * (walk_steps + diag_steps) / (head["ms_per_step"] * 1e-3),
        "walk": {"ms": head["walk_ms"], "prepare_ms": head["prepare_ms"],
                 "merge_steps_per_s": walk_rate},
        "gpu_launches": head["steps"] * step_launches(prec, args.layout),
        "e2e": {"value": units * pairs / e2e_s, "unit": "pair-integrals/s",
                "h2d_bytes_per_step": world * h2d, "d2h_bytes_per_step": world * d2h,
                "ms_per_step": e2e_s * 1e3,
                "phases_ms": dict(zip(("h2d", "prepare_walk_and_d2h"),
                                      np.mean(np.array(phases), axis=0).round(3).tolist())),
                "d2h": ("rows streamed to pinned host memory by a copy kernel on a second "
                        "stream while later bands of the walk run" if not split else
                        "each rank reads back its whole matrices after its shard")},
        "pipe_peaks": pp,
        "clocks": head["clocks"],
    }
    if walk_rate is not None:
        line["roofline"] = {
            "bound": "alu", "achieved": walk_rate, "peak": issue_peak,
            "unit": "merge-steps/s", "frac": walk_rate / issue_peak,
            "traffic": (TRAFFIC_RECORD["by_schedule_layout"].get((head["schedule"], args.layout))
                        if (walk_source_id() == TRAFFIC_RECORD["source_sha256_16"]
                            and N == 20000) else None),
            "traffic_unit": "DRAM bytes per walk launch (ncu)",
            "peak_basis": f"{sms} SMs x 128 lanes x {fmax/1e6:.0f} MHz / {tally(prec)} "
                          "ops per merge step (fused L1+L2+Gram tally; exact float64 "
                          "comparisons by order keys)"}
    if sorted_walk is not None:
        line["sorted_output"] = {"walk_ms": sorted_walk,
                                 "traffic": (TRAFFIC_RECORD["by_schedule_layout"].get(
                                     (head["schedule"], "sorted"))
                                     if walk_source_id() == TRAFFIC_RECORD["source_sha256_16"]
                                     and N == 20000 else None),
                                 "merge_steps_per_s": walk_steps / (sorted_walk * 1e-3),
                                 "note": "layout PCF_OUT_FULL_SORTED: same walk, matrices in "
                                         "the library's sort order (perm from pcf_sort_order)"}

    def side(name, note, bound="alu"):
        f = results[name]
        wr = walk_steps / (f["walk_ms"] * 1e-3)
        if bound == "alu":
            pk = sms * 128 * fmax / tally(name)
            basis = f"tally {tally(name)} ops per merge step"
        else:
            r64 = pp["fp64"]["lane_ops_per_clk_per_sm"]
            pk = sms * r64 * fmax / FP64_OPS_PER_STEP
            basis = (f"{sms} SMs x {r64:.2f} FP64 lane-ops/clk x {fmax/1e6:.0f} MHz / "
                     f"{FP64_OPS_PER_STEP} FP64 ops per step")
        d = {"value": units * pairs / (f["ms_per_step"] * 1e-3), "unit": "pair-integrals/s",
             "ms_per_step": f["ms_per_step"], "walk_ms": f["walk_ms"], "prepare_ms": f["prepare_ms"],
             "merge_steps_per_s": wr, "schedule": f["schedule"],
             "roofline": {"bound": bound, "achieved": wr, "peak": pk, "unit": "merge-steps/s",
                          "frac": wr / pk, "peak_basis": basis}}
        if note:
            d["note"] = note
        return d

    if not split:
        if "f32b" in results and prec != "f32b":
            line["f32b"] = side("f32b", "float32 walk, FMA block sums of <= 16 rectangles, Kahan "
                                        "across blocks (error <= ~18u sum|terms|)")
        if "f32c_round" in results and prec != "f32c_round":
            line["f32c_round"] = side("f32c_round", "opt-in PCF_PREC_ROUND_TIMES: float64 times "
                                                    "rounded to float32 when packed (8-byte "
                                                    "elements; comparisons and widths on the "
                                                    "rounded times)")
        if "f64" in results:
            line["fp64"] = side("f64", None, bound="fp64 pipe")
    if not args.no_cpu and world == 1:
        rec, want, diag = cpu_baseline(s)
        line["cpu_baseline"] = rec
        if samples:
            nrows = min(want["l1"].shape[0], check_rows[1] - check_rows[0])
            err = {}
            for name, got in samples.items():
                err[name] = matrix_errors({m: got[m][:nrows] for m in METRICS},
                                          {m: want[m][:nrows] for m in METRICS}, diag,
                                          SAMPLE_ROW0)
            line["error"] = {
                "vs": "float64 oracle walk", "rows": f"{SAMPLE_ROW0}..{SAMPLE_ROW0 + nrows} x all "
                                                    f"{N} columns",
                "measure": "distances max |x - x*| / |x*|; Gram max |x - x*| / sqrt(G*_ii G*_jj)",
                "output_dtype": "float32 (its rounding, <= 6e-8, is included)",
                "by_form": err}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------------
# Other workloads (one JSON line each): python bench.py --workload NAME|all
# --------------------------------------------------------------------------
def _timed(step, steps, warmup, flush, stream):
    """Per-step device time (ms) with CUDA events; L2 flushed before each."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _cpu_rows(a, metrics, b=None, seconds_target=8.0, row0=0, p=None):
    """Oracle on all host cores over a row block sized to ~seconds_target."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    ncols = a.n if b is None else b.n
    rows = 2
    t0 = time.perf_counter()
    oracle.matrix(a, b, metric=metrics[0], p=p or 1.0, rows=(row0, row0 + rows), nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    rows = int(max(2, min(a.n - row0, rows * seconds_target / (dt * len(metrics)))))
    t0 = time.perf_counter()
    for m in metrics:
        mm, pp = (m, None) if isinstance(m, str) else (m[0], m[1])
        oracle.matrix(a, b, metric=mm, p=pp or 1.0, rows=(row0, row0 + rows), nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": len(metrics) * rows * ncols / dt, "unit": "pair-integrals/s",
            "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": f"rows {row0}..{row0 + rows} x all {ncols} columns x {len(metrics)} "
                      "metrics, float64 oracle walk, one thread per core"}


def _clip_after(s, t_end):
    """Breakpoints of each PCF before t_end, plus one at t_end (the moved
    collection of a weight that vanishes after t_end has this shape)."""
    offs, ts, vs = [0], [], []
    for i in range(s.n):
        t, v = s.pcf(i)
        keep = t < t_end
        ts.append(np.append(t[keep], t_end))
        vs.append(np.append(v[keep], 0.0))
        offs.append(offs[-1] + ts[-1].size)
    return np.array(offs, np.int64), np.concatenate(ts), np.concatenate(vs)


def _cpu_rows_weighted(a, w, seconds_target=8.0, row0=1000):
    """The oracle's weighted walk (one row per pool task) on a row sample."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cores = len(os.sched_getaffinity(0))

    def row(i):
        tf, vf = a.pcf(i)
        for j in range(a.n):
            for m, p in (("l1", 1.0), ("l2", 2.0), ("gram", 1.0)):
                oracle.integral_w(tf, vf, *a.pcf(j), *w, m, p)

    t0 = time.perf_counter()
    row(row0)
    dt = max(time.perf_counter() - t0, 1e-3)
    rows = int(max(1, min(64, seconds_target / dt)))
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(row, range(row0, row0 + rows)))
    dt = time.perf_counter() - t0
    return {"value": 3 * rows * a.n / dt, "unit": "pair-integrals/s", "cores": cores,
            "kind": "oracle", "seconds": dt,
            "sample": f"rows {row0}..{row0 + rows} x all {a.n} columns x 3 metrics, float64 "
                      "three-list walk called pair by pair from Python threads"}


def _line(name, value, unit, ms, steps, warmup, dtype, config, **extra):
    d = {"metric": "pair-integrals/s and merge-steps/s at 1 GB300 (FP32-comp vs FP64), "
                   "% issue roofline",
         "workload": name, "value": value, "unit": unit, "n_gpus": 1, "steps": steps,
         "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}
    d.update(extra)
    return d


# secondary workloads that split over several ranks (the others are one-GPU
# measurements and are skipped under torchrun)
MULTI_RANK_WORKLOADS = ("gradient",)


def dist_world():
    return dist_env()[1]


def run_workload(name, args):
    import torch
    import paper_2404_07183_gb300 as P
    P.build.build()
    rank, world, local = dist_env()
    dev = f"cuda:{local}"
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        assert name in MULTI_RANK_WORKLOADS, name
        if not dist.is_initialized():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    pp = pipe_peaks()
    sms = pp["sms"]
    fmax = float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6
    issue = lambda tally: sms * 128 * fmax / tally
    fp64 = lambda ops: sms * pp["fp64"]["lane_ops_per_clk_per_sm"] * fmax / ops

    if name == "uniform_small":
        s = synth.uniform_small()
        N = s.n
        steps_walk, _ = exact_walk_steps(s)
        x = P.PcfTensors.from_numpy(s, dev)
        pairs = N * (N - 1) // 2
        out = {}
        tuned = {}
        from paper_2404_07183_gb300 import autotune
        for prec in ("f64", "f32c"):
            o = [torch.empty((N, N), dtype=torch.float64, device=dev)]
            ws = torch.empty(P.pcf_workspace_size(x, None, prec), dtype=torch.uint8, device=dev)
            sched, timings = autotune.tune_pairwise(x, ["l1"], prec, out_dtype=torch.float64,
                                                    repeats=3)
            tuned[prec] = {"schedule": sched, "timings_ms": timings}

            def step():
                P.pcf_prepare(x, prec, workspace=ws)
                P.pcf_pairwise(x, ["l1"], precision=prec, out=o, workspace=ws, prepared=True,
                               check=False, schedule=tuned[prec]["schedule"])
            step()
            P.pcf_check(ws)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            ms = _timed(g.replay, args.steps, args.warmup, flush, stream)
            P.pcf_check(ws)
            out[prec] = float(np.mean(ms))
        ms = out["f64"]
        rate = steps_walk / (ms * 1e-3)
        return _line(name, pairs / (ms * 1e-3), "pair-integrals/s", ms, args.steps, args.warmup,
                     "f64", {"workload": "uniform_small N=1000 n~U{10..100} Exp(1) N(0,1) "
                             "float64, L1 upper triangle", "N": N, "pairs": pairs,
                             "merge_steps": steps_walk, "cuda_graph": True,
                             "l2": "flushed between steps", "autotune": tuned},
                     merge_steps_per_s=rate,
                     roofline={"bound": "fp64 pipe", "achieved": rate, "peak": fp64(3),
                               "unit": "merge-steps/s", "frac": rate / fp64(3),
                               "note": "whole step (prepare + walk, 6 launches in one graph)"},
                     f32c={"ms_per_step": out["f32c"], "value": pairs / (out["f32c"] * 1e-3)},
                     cpu_baseline=_cpu_rows(s, ["l1"], seconds_target=4.0))

    if name == "lognormal":
        s = synth.lognormal(n_pcfs=args.n or 100000)
        N = s.n
        steps_walk, diag = exact_walk_steps(s)
        x = P.PcfTensors.from_numpy(s, dev)
        pairs = N * (N + 1) // 2
        o = [torch.empty((pairs,), dtype=torch.float32, device=dev)]
        res = {}
        from paper_2404_07183_gb300 import autotune
        if args.schedule:
            sched, tune_ms = args.schedule, None
        else:
            sched, tune_ms = autotune.tune_pairwise(x, ["gram"], "f32c", layout="upper", repeats=1)
        scheds = {"f32c": sched, "f32": sched}
        if args.schedule:
            scheds["f64"] = args.schedule
        else:
            # the float64 walk is bound by the FP64 pipe, not by issue: its own
            # choice between the 512-thread schedules (one timed call each)
            scheds["f64"], _ = autotune.tune_pairwise(
                x, ["gram"], "f64", layout="upper", repeats=1,
                candidates=(("tile512x2", 0), ("tile512x3", 0)))
        for prec in ("f32c", "f32", "f64"):
            ws = torch.empty(P.pcf_workspace_size(x, None, prec), dtype=torch.uint8, device=dev)
            mids = []

            def step():
                P.pcf_prepare(x, prec, workspace=ws)
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                mids.append(e)
                P.pcf_pairwise(x, ["gram"], precision=prec, layout="upper", out=o, workspace=ws,
                               prepared=True, check=False, schedule=scheds[prec])
            # the float64 walk takes ~10 s per step at full size: one timed step
            nst = 1 if prec == "f64" else max(1, min(args.steps, 2))
            ms = _timed(step, nst, 1, flush, stream)
            P.pcf_check(ws)
            res[prec] = float(np.mean(ms))
            del ws
        ms = res["f32c"]
        # float64 operations per merge step of the Gram walk: dt, a*b, fma
        gram64_ops = 3
        rate = (steps_walk + diag) / (ms * 1e-3)
        tally = 5 + 2 + 3
        return _line(name, pairs / (ms * 1e-3), "pair-integrals/s", ms, max(1, min(args.steps, 2)),
                     1, "f32 (compensated)",
                     {"workload": "lognormal N=100000 n=clip(round(LogNormal(ln100,1)),2,10000) "
                                  "Exp(1) N(0,1) float32, L2 Gram upper triangle (packed, f32)",
                      "N": N, "nnz": s.nnz, "max_len": int(s.lengths().max()), "pairs": pairs,
                      "merge_steps": steps_walk + diag, "l2": "flushed between steps",
                      "schedule": sched, "autotune_ms": tune_ms},
                     merge_steps_per_s=rate,
                     roofline={"bound": "alu", "achieved": rate, "peak": issue(tally),
                               "unit": "merge-steps/s", "frac": rate / issue(tally),
                               "note": f"whole step; tally {tally} ops/step (Gram, Kahan)"},
                     f32={"ms_per_step": res["f32"], "value": pairs / (res["f32"] * 1e-3),
                          "frac": (steps_walk + diag) / (res["f32"] * 1e-3) / issue(5 + 2)},
                     fp64={"ms_per_step": res["f64"], "value": pairs / (res["f64"] * 1e-3),
                           "merge_steps_per_s": (steps_walk + diag) / (res["f64"] * 1e-3),
                           "frac": (steps_walk + diag) / (res["f64"] * 1e-3) / fp64(gram64_ops),
                           "bound": "fp64 pipe", "schedule": scheds["f64"],
                           "note": f"{gram64_ops} float64 ops per merge step (dt, a*b, fma); "
                                   "one timed step"},
                     cpu_baseline=(None if args.no_cpu else
                                   _cpu_rows(s, ["gram"], seconds_target=8.0, row0=N // 2)))

    if name == "appendix_a":
        s = synth.appendix_a(n_pcfs=args.n or 50000)
        N = s.n
        steps_walk, _ = exact_walk_steps(s)
        x = P.PcfTensors.from_numpy(s, dev)
        pairs = N * (N - 1) // 2
        o = [torch.empty((N, N), dtype=torch.float32, device=dev)]
        from paper_2404_07183_gb300 import autotune
        res = {}
        for prec in ("f32c", "f32", "f64", "f32c_round"):
            if args.schedule:
                sched = args.schedule
            else:
                sched, _ = autotune.tune_pairwise(x, ["l1"], prec, repeats=1,
                                                  candidates=(("tile1024", 0), ("tile512x2", 0)))
            ws = torch.empty(P.pcf_workspace_size(x, None, prec), dtype=torch.uint8, device=dev)

            def step():
                P.pcf_prepare(x, prec, workspace=ws)
                P.pcf_pairwise(x, ["l1"], precision=prec, out=o, workspace=ws, prepared=True,
                               check=False, schedule=sched)
            ms = float(np.mean(_timed(step, 1, 1, flush, stream)))
            P.pcf_check(ws)
            res[prec] = {"ms_per_step": ms, "value": pairs / (ms * 1e-3),
                         "merge_steps_per_s": steps_walk / (ms * 1e-3), "schedule": sched}
            del ws
        ms = res["f32c"]["ms_per_step"]
        rate = steps_walk / (ms * 1e-3)
        return _line(name, pairs / (ms * 1e-3), "pair-integrals/s", ms, 1, 1, "f32 (compensated)",
                     {"workload": f"appendix_a N={N}: n~U{{10..1000}}, times |alpha|*sorted|t~|, "
                                  "N(0,1) values, final 0 (float64 input), L1 distance matrix, "
                                  "full N x N float32",
                      "N": N, "pairs": pairs, "merge_steps": steps_walk,
                      "paper_context": "L1 on 500,000 such PCFs: ~423 s on 8 A100 "
                                       "(~3.7e7 pair-integrals/s per GPU, precision not stated)"},
                     merge_steps_per_s=rate,
                     roofline={"bound": "alu", "achieved": rate, "peak": issue(5 + 1 + 4 + KEYED_EXTRA),
                               "unit": "merge-steps/s",
                               "frac": rate / issue(5 + 1 + 4 + KEYED_EXTRA),
                               "note": "whole step; tally 13 ops/step (L1, Kahan, exact float64 "
                                       "comparisons by order keys)"},
                     forms=res,
                     cpu_baseline=_cpu_rows(s, ["l1"], seconds_target=8.0, row0=N // 3))

    if name == "weighted":
        # the stable-rank workload against a PCF weight: a decaying step
        # weight w = 1, 1/2, 1/4, ... on [0, 5), [5, 10), ..., 0 after 40 (the
        # curves' features near the start count more; compact support)
        s = workload(0, args.n)
        N = s.n
        tw = np.arange(0.0, 45.0, 5.0)
        vw = np.concatenate([0.5 ** np.arange(8), [0.0]])
        x = P.PcfTensors.from_numpy(s, dev)
        pairs = 2 * (N * (N - 1) // 2) + N * (N + 1) // 2
        outs = [torch.empty((N, N), dtype=torch.float32, device=dev) for _ in METRICS]
        # merge steps of the moved collection: the weight leaves the breakpoints
        # of [0, 40) and drops those after 40 (a zero-valued end at W(inf))
        cut = synth.PcfSet(*_clip_after(s, 40.0))
        steps_walk, diag_steps = exact_walk_steps(cut)
        res = {}
        for prec in ("f32c", "f64"):
            sched = args.schedule or ("tile512x2" if prec == "f32c" else "tile1024")
            ws = torch.empty(P.pcf_weighted_workspace_size(x, (tw, vw), prec), dtype=torch.uint8,
                             device=dev)

            def step():
                P.pcf_pairwise_weighted(x, (tw, vw), METRICS, precision=prec, out=outs,
                                        workspace=ws, check=False, schedule=sched)
            ms = _timed(step, max(1, min(args.steps, 3)), 1, flush, stream)
            P.pcf_check(ws)
            res[prec] = {"ms_per_step": float(np.mean(ms)), "schedule": sched}
            del ws
        ms = res["f32c"]["ms_per_step"]
        rate = (steps_walk + diag_steps) / (ms * 1e-3)
        tally = TALLY["f32c"] + KEYED_EXTRA
        r64 = (steps_walk + diag_steps) / (res["f64"]["ms_per_step"] * 1e-3)
        cpu = _cpu_rows_weighted(s, (tw, vw), seconds_target=8.0)
        return _line(name, pairs / (ms * 1e-3), "pair-integrals/s", ms,
                     max(1, min(args.steps, 3)), 1, "f32 (compensated)",
                     {"workload": f"stable_rank N={N} against the PCF weight 2^-k on "
                                  "[5k, 5k+5), k = 0..7, 0 after 40: L1+L2+Gram fused, "
                                  "full N x N float32",
                      "N": N, "pairs": pairs, "merge_steps": steps_walk + diag_steps,
                      "step": "move the breakpoints to W(t) (compacted, float64) + prepare + "
                              "walk, one pcf_pairwise_weighted call"},
                     merge_steps_per_s=rate,
                     roofline={"bound": "alu", "achieved": rate, "peak": issue(tally),
                               "unit": "merge-steps/s", "frac": rate / issue(tally),
                               "note": f"whole step; tally {tally} ops/step (fused L1+L2+Gram, "
                                       "Kahan, order keys)"},
                     fp64={"value": pairs / (res["f64"]["ms_per_step"] * 1e-3),
                           "ms_per_step": res["f64"]["ms_per_step"], "merge_steps_per_s": r64,
                           "roofline": {"bound": "fp64 pipe", "achieved": r64,
                                        "peak": fp64(FP64_OPS_PER_STEP),
                                        "frac": r64 / fp64(FP64_OPS_PER_STEP)}},
                     forms=res, cpu_baseline=cpu)

    if name == "segments":
        s = synth.lognormal(n_pcfs=args.n or 100000)
        N = s.n
        x = P.PcfTensors.from_numpy(s, dev)
        out = torch.empty(N, dtype=torch.float64, device=dev)
        ws = torch.empty(P.pcf_workspace_size(x, None, "f64"), dtype=torch.uint8, device=dev)

        def step(prec):
            P.pcf_segment_integrals(x, "lp", 2.0, True, precision=prec, out=out, workspace=ws,
                                    check=False)
            P.pcf_segment_integrals(x, "integral", precision=prec, out=out, workspace=ws,
                                    check=False)

        def graphed(prec):
            step(prec)
            P.pcf_check(ws)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step(prec)
            return g
        # device time: the two calls replayed from a CUDA graph (no host gaps);
        # direct: the same calls issued from Python one by one
        g32, g64 = graphed("f32c"), graphed("f64")
        ms = float(np.mean(_timed(g32.replay, args.steps, args.warmup, flush, stream)))
        ms64 = float(np.mean(_timed(g64.replay, args.steps, args.warmup, flush, stream)))
        ms_direct = float(np.mean(_timed(lambda: step("f32c"), args.steps, args.warmup, flush,
                                         stream)))
        P.pcf_check(ws)
        seg_per_s = 2 * s.nnz / (ms * 1e-3)
        hbm = float(measured_peaks().get("hbm_gbs", 6800.0)) * 1e9
        bytes_per_call = s.nnz * 2 * 4 + (N + 1) * 8 + N * 8 + N * 8
        fp64_rate = fp64(3)             # dt, h, fma per segment
        import oracle
        t0 = time.perf_counter()
        k = 0
        for i in range(0, N, 10):
            t, v = s.pcf(i)
            oracle.segment_integral(t, v, "lp", 2.0)
            oracle.segment_integral(t, v, "integral")
            k += 2 * t.size
        dt = time.perf_counter() - t0
        return _line(name, 2 * N / (ms * 1e-3), "PCF-integrals/s", ms, args.steps, args.warmup,
                     "f32 (Kahan per segment)",
                     {"workload": "segment iteration over the lognormal set N=100000 "
                                  "(16.5M breakpoints): L2 norms and plain integrals over [0, inf)",
                      "N": N, "nnz": s.nnz, "l2": "flushed between steps",
                      "timing": "CUDA graph replay of both calls (device time)"},
                     direct_call_ms=ms_direct,
                     segments_per_s=seg_per_s,
                     roofline={"bound": "hbm", "achieved": 2 * bytes_per_call / (ms * 1e-3) / 1e9,
                               "peak": hbm / 1e9, "unit": "GB/s",
                               "frac": (2 * bytes_per_call / (ms * 1e-3)) / hbm,
                               "traffic": None,
                               "note": "input bytes (times, values, offsets) + outputs per call; "
                                       "the input check runs on the same loads"},
                     f64={"ms_per_step": ms64, "segments_per_s": 2 * s.nnz / (ms64 * 1e-3),
                          "fp64_frac": (2 * s.nnz / (ms64 * 1e-3)) / fp64_rate},
                     cpu_baseline={"value": k / 2 / dt * (2 * N) / (2 * s.nnz) if dt else None,
                                   "unit": "PCF-integrals/s", "cores": 1, "kind": "oracle",
                                   "seconds": dt,
                                   "sample": "every 10th PCF, both functionals, one thread"})

    if name == "reduce":
        from paper_2404_07183_gb300 import api
        s = synth.stable_rank(n_pcfs=args.n or 20480)
        N = s.n
        x = P.PcfTensors.from_numpy(s, dev)
        hbm = float(measured_peaks().get("hbm_gbs", 6800.0)) * 1e9
        forms = {}
        for red, m in (("mean", 128), ("std", 16)):
            std_rows = x.nnz + m * P.pcf_reduce(x, m, "mean").nnz if red == "std" else 0
            ws = torch.empty(api.pcf_reduce_workspace_size(x, m, red, std_rows),
                             dtype=torch.uint8, device=dev)
            out = api._csr_out(N // m, x.nnz, dev)

            def step():
                P.pcf_reduce(x, m, red, workspace=ws, check=False, trim=False, out=out)
            step()
            P.pcf_check(ws)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            ms = float(np.mean(_timed(g.replay, args.steps, args.warmup, flush, stream)))
            ms_direct = float(np.mean(_timed(step, args.steps, args.warmup, flush, stream)))
            P.pcf_check(ws)
            pos, rows = api.pcf_reduce_counters(ws)
            alg = 16 * s.nnz + 16 * (pos + rows)
            forms[red] = {"group_size": m, "ms_per_step": ms, "direct_call_ms": ms_direct,
                          "breakpoints_per_s": s.nnz / (ms * 1e-3),
                          "merge_positions": pos, "rows_written": rows,
                          "merge_positions_per_s": pos / (ms * 1e-3),
                          "hbm_frac": alg / (ms * 1e-3) / hbm,
                          "result_rows": int(out[1][-1].item())}
        import oracle
        t0 = time.perf_counter()
        sub = synth.subset(s, np.arange(16 * 128))
        oracle.reduce(sub, 128, "mean")
        sub_std = synth.subset(s, np.arange(64 * 16))
        oracle.reduce(sub_std, 16, "std")
        dt = time.perf_counter() - t0
        cores = len(os.sched_getaffinity(0))
        f = forms["mean"]
        return _line(name, f["breakpoints_per_s"], "input-breakpoints/s", f["ms_per_step"],
                     args.steps, args.warmup, "f64",
                     {"workload": f"mean of {N // 128} groups of 128 stable-rank PCFs "
                                  f"(N={N}, {s.nnz} breakpoints) by binary ReducePair trees; "
                                  "std of groups of 16 alongside",
                      "N": N, "nnz": s.nnz, "l2": "flushed between steps",
                      "timing": "CUDA graph replay of one call (device time)"},
                     roofline={"bound": "hbm",
                               "achieved": (16 * s.nnz + 16 * (f["merge_positions"]
                                                               + f["rows_written"]))
                               / (f["ms_per_step"] * 1e-3) / 1e9,
                               "peak": hbm / 1e9, "unit": "GB/s", "frac": f["hbm_frac"],
                               "traffic": None,
                               "note": "16 B per input row read once, plus 16 B per merge "
                                       "position and per row written over all ReducePair passes "
                                       "(library work counters); the call also validates"},
                     forms=forms,
                     cpu_baseline={"value": (sub.nnz + sub_std.nnz) / dt,
                                   "unit": "input-breakpoints/s", "cores": cores,
                                   "kind": "oracle", "seconds": dt,
                                   "sample": "mean of 16 groups of 128 and std of 64 groups "
                                             "of 16, all host threads"})

    if name == "gradient":
        s, G = synth.gradient(n_pcfs=args.n or 4096)
        N = s.n
        steps_walk, diag = exact_walk_steps(s)
        x = P.PcfTensors.from_numpy(s, dev)
        Gt = torch.from_numpy(G).to(dev)
        pairs = N * (N - 1) // 2
        # several ranks (torchrun): each walks its strided share of the tiles
        # and one NCCL sum all-reduce of the two gradient arrays gives every
        # rank the whole gradient
        world = dist_world()
        shard = (dist_env()[0], world) if world > 1 else None

        def step():
            gv, gt = P.pcf_pairwise_backward(x, ("l2", False), Gt, check=False, shard=shard)
            if world > 1:
                import torch.distributed as dist
                dist.all_reduce(gv)
                dist.all_reduce(gt)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()
        ms = float(np.mean(_timed(step, args.steps, args.warmup, flush, stream)))
        if world > 1:
            # every timed step ends in the all-reduce, so the ranks finish
            # together; the slowest rank's mean is the step time
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        rate = steps_walk / (ms * 1e-3)
        import oracle
        sub = synth.subset(s, np.arange(300))
        t0 = time.perf_counter()
        if not args.no_cpu and rank == 0:
            oracle.backward(sub, G[:300, :300], metric="l2", p=2.0)
        dt = max(time.perf_counter() - t0, 1e-9)
        # float64 operations per rectangle of the L2 adjoint: dt, d, d*dt, two
        # value-gradient fma; time gradient of the advancing side: v_new - v_other,
        # its square, fma(d, d, -b*b), times the weight
        bw_ops = 9
        cfg = {"workload": "gradient N=4096 n~U{20..200} Exp(1) N(0,1) float64, "
                           "d(sum G*D2^2)/d(values, times)", "N": N, "pairs": pairs,
               "merge_steps": steps_walk, "l2": "flushed between steps"}
        extra = {}
        if world > 1:
            cfg["parallelism"] = f"tile shards over {world} ranks + NCCL sum all-reduce of the gradients"
            extra = {"n_gpus": world, "scaling": "strong"}
        return _line(name, pairs / (ms * 1e-3), "pair-gradients/s", ms, args.steps, args.warmup,
                     "f64", cfg, merge_steps_per_s=rate,
                     roofline={"bound": "fp64 pipe", "achieved": rate,
                               "peak": fp64(bw_ops) * world,
                               "unit": "merge-steps/s", "frac": rate / (fp64(bw_ops) * world),
                               "note": f"whole backward call (recomputing walk + scatter"
                                       f"{' + all-reduce' if world > 1 else ''}); "
                                       f"{bw_ops} float64 ops per merge step"
                                       f"{f', peak of {world} GPUs' if world > 1 else ''}"},
                     **extra,
                     cpu_baseline={"value": 300 * 299 / 2 / dt, "unit": "pair-gradients/s",
                                   "cores": 1, "kind": "oracle", "seconds": dt,
                                   "sample": "first 300 PCFs, single-threaded oracle adjoint"})

    if name == "euler":
        a, b = synth.euler()
        NA, NB = a.n, b.n
        xa = P.PcfTensors.from_numpy(a, dev)
        xb = P.PcfTensors.from_numpy(b, dev)
        metrics = [("lp", 1.0), ("lp", 2.0), ("lp", 3.0)]
        block = 2048
        nblk = (NA + block - 1) // block
        bufs = [[torch.empty((block, NB), dtype=torch.float32, device=dev) for _ in metrics]
                for _ in range(2)]
        host = [torch.empty((block, NB), dtype=torch.float32).pin_memory() for _ in metrics]
        copy = torch.cuda.Stream()
        done = [torch.cuda.Event(), torch.cuda.Event()]
        ws = torch.empty(P.pcf_workspace_size(xa, xb, "f32c"), dtype=torch.uint8, device=dev)

        def sweep():
            for k in range(nblk):
                r0, r1 = k * block, min(NA, (k + 1) * block)
                buf = bufs[k % 2]
                stream.wait_event(done[k % 2])
                views = [t[: r1 - r0] for t in buf]
                P.pcf_cross(xa, xb, r0, r1, metrics, precision="f32c", out=views, workspace=ws,
                            reuse_b=k > 0, check=False)
                ev = torch.cuda.Event()
                ev.record(stream)
                copy.wait_event(ev)
                with torch.cuda.stream(copy):
                    for h, v in zip(host, views):
                        h[: r1 - r0].copy_(v, non_blocking=True)
                    done[k % 2].record(copy)
            stream.wait_stream(copy)
        ms = float(np.mean(_timed(sweep, 1, 1, flush, stream)))
        pairs = NA * NB
        # |T_i u T_j| = n_i + n_j - 1 - (shared positive times); a time held by
        # cA PCFs of A and cB PCFs of B is shared by cA * cB pairs
        ta, ca = np.unique(np.asarray(a.times[a.times > 0], np.float64), return_counts=True)
        tb, cb = np.unique(np.asarray(b.times[b.times > 0], np.float64), return_counts=True)
        _, ia, ib = np.intersect1d(ta, tb, assume_unique=True, return_indices=True)
        shared = int(np.sum(ca[ia].astype(np.int64) * cb[ib].astype(np.int64)))
        steps_walk = NB * a.nnz + NA * b.nnz - pairs - shared
        rate = steps_walk / (ms * 1e-3)
        tally = 5 + 1 + (1 + 3) + (2 + 3) + (3 + 3)
        return _line(name, 3 * pairs / (ms * 1e-3), "pair-integrals/s", ms, 1, 1,
                     "f32 (compensated)",
                     {"workload": "euler A x B 50000 x 50000, n=1000, integer steps +-1..3 at "
                                  "Exp(1) times, float32; L1+L2+L3 fused, row blocks of 2048 "
                                  "double-buffered with async D2H to pinned host",
                      "pairs": pairs, "merge_steps": steps_walk, "blocks": nblk,
                      "d2h_bytes_per_step": 3 * pairs * 4},
                     merge_steps_per_s=rate,
                     roofline={"bound": "alu", "achieved": rate, "peak": issue(tally),
                               "unit": "merge-steps/s", "frac": rate / issue(tally),
                               "note": f"whole sweep incl. packing per block; tally {tally}"},
                     cpu_baseline=_cpu_rows(a, ["l1", "l2", ("lp", 3.0)], b=b, seconds_target=8.0))
    raise SystemExit(f"unknown workload {name}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32c",
                    choices=["f32c", "f32b", "f32", "f64", "f32c_round", "f32b_round", "f32_round"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-rows", type=int, default=48)
    ap.add_argument("--n", type=int, default=None,
                    help="smaller stable-rank collection (profiling runs); default 20000")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs: an independent batch per GPU (weak scaling) "
                         "instead of one matrix split over them")
    ap.add_argument("--check-rows", type=int, default=256,
                    help="rows of every form's matrices compared with the oracle's")
    ap.add_argument("--layout", default="full", choices=["full", "sorted"],
                    help="output layout of the timed walk (profiling runs)")
    ap.add_argument("--schedule", default=None,
                    choices=["tile1024", "tile512x2", "tile512x3", "mergepath", "auto"],
                    help="force a walk schedule instead of autotuning it")
    ap.add_argument("--workload", default="stable_rank",
                    choices=["stable_rank", "uniform_small", "lognormal", "gradient", "euler",
                             "appendix_a", "weighted", "segments", "reduce", "all"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    try:
        import torch
        ndev = torch.cuda.device_count()
    except Exception:
        ndev = 0
    action, what = resolve_launch(args.gpus, os.environ, ndev)
    if action == "error":
        print(json.dumps({"error": what}), flush=True)
        sys.exit(2)
    if action == "spawn":
        import random
        cmd = spawn_command(what, sys.argv[1:], 29500 + random.randrange(1000))
        sys.exit(subprocess.call(cmd))
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "stable_rank":
        run_ours(args)
    else:
        names = (["uniform_small", "gradient", "lognormal", "euler", "appendix_a", "weighted",
                  "segments", "reduce"]
                 if args.workload == "all"
                 else [args.workload])
        rank, world, _ = dist_env()
        if world > 1:
            names = [nm for nm in names if nm in MULTI_RANK_WORKLOADS]
            if not names:
                if rank == 0:
                    print(json.dumps({"error": f"--workload {args.workload} runs on one GPU; "
                                               "with several GPUs the headline and the "
                                               "gradient workloads split their work"}), flush=True)
                sys.exit(2)
        for nm in names:
            d = None
            if rank != 0:
                run_workload(nm, args)
                continue
            # clocks sampled over the whole workload run (its timed steps are
            # too short for the 200 ms sampling period alone)
            clk_path = os.path.join(tempfile.gettempdir(), f"pcf_bench_clocks_{nm}.csv")
            os.makedirs(os.path.dirname(clk_path), exist_ok=True)
            sampler, sfh = start_clock_sampler(clk_path)
            d = run_workload(nm, args)
            d["clocks"] = stop_clock_sampler(sampler, sfh, clk_path, 0) if sampler else None
            if d["clocks"] is not None:
                d["clocks"]["window"] = "whole workload run"
            print(json.dumps(d), flush=True)
        if world > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    main()
