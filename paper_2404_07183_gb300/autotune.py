"""Autotuner for the walk's work decomposition.

For a class of inputs (GPU, precision, metric set, layout, and the binned
size N, mean and maximum PCF length), it times every candidate schedule of
``pcf_pairwise_ex`` on the actual collection -- 32 x 32 tiles with one
1024-thread CTA per SM, the same tiles with two 512-thread CTAs per SM, and
the warp-per-pair merge path -- and remembers the fastest in a JSON cache
(``$PCF_GB300_TUNE_CACHE`` or ``~/.cache/pcf_gb300/tune.json``).  Later
calls in the same class use the cached schedule without timing again.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import api

CANDIDATES = (("tile1024", 0), ("tile512x2", 0), ("tile512x3", 0), ("mergepath", 0))
_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("PCF_GB300_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "pcf_gb300", "tune.json")


def _bucket(v: float) -> int:
    return int(math.floor(math.log2(max(float(v), 1.0))))


def input_class(n: int, lengths_mean: float, lengths_max: int, metrics, precision, layout,
                gpu: str) -> str:
    ms = ",".join(sorted(str(api.parse_metric(m)[:2]) for m in metrics))
    return (f"{gpu}|{precision}|{layout}|{ms}|N{_bucket(n)}|mean{_bucket(lengths_mean)}"
            f"|max{_bucket(lengths_max)}")


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path=None) -> None:
    path = path or cache_path()
    with _lock:
        cache = load_cache(path)
        cache[key] = entry
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def choose(timings: dict) -> str:
    """Fastest candidate name from {name: milliseconds}."""
    return min(timings, key=lambda k: timings[k])


def _class_of(x: api.PcfTensors, metrics, precision, layout) -> str:
    lens = (x.offsets[1:] - x.offsets[:-1])
    mean = float(lens.double().mean().item()) if x.n else 1.0
    mx = int(lens.max().item()) if x.n else 1
    # float64 input walked in float32 runs the keyed form (16-byte elements),
    # float32 input the 8-byte form: different best schedules
    prec_form = f"{precision}/{str(x.times.dtype).replace('torch.', '')}"
    return input_class(x.n, mean, mx, metrics, prec_form, layout,
                       torch.cuda.get_device_name(x.times.device))


def tune_pairwise(x: api.PcfTensors, metrics, precision="f32c", layout="full",
                  out_dtype=torch.float32, repeats=2, path=None, candidates=CANDIDATES):
    """Time every candidate on ``x`` and cache the fastest; returns (name, timings)."""
    ws = api.pcf_prepare(x, precision)
    api.pcf_check(ws)
    n = x.n
    # the merge path only pays when the tiles cannot occupy the GPU
    nb = (n + 31) // 32
    sms = torch.cuda.get_device_properties(x.times.device).multi_processor_count
    if nb * (nb + 1) // 2 >= 2 * sms:
        candidates = tuple(c for c in candidates if c[0] != "mergepath") or candidates
    shape = (n * (n + 1) // 2,) if layout == "upper" else (n, n)
    outs = [torch.empty(shape, dtype=out_dtype, device=x.times.device) for _ in metrics]
    stream = torch.cuda.current_stream()
    timings = {}
    for name, window in candidates:
        sched = (name, window)
        api.pcf_pairwise(x, metrics, precision, layout, out=outs, workspace=ws, prepared=True,
                         check=False, schedule=sched)
        best = float("inf")
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            api.pcf_pairwise(x, metrics, precision, layout, out=outs, workspace=ws,
                             prepared=True, check=False, schedule=sched)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        timings[name] = best
    api.pcf_check(ws)
    name = choose(timings)
    store(_class_of(x, metrics, precision, layout), {"schedule": name, "timings_ms": timings},
          path)
    return name, timings


def schedule_for(x: api.PcfTensors, metrics, precision="f32c", layout="full", tune=True,
                 path=None, **kw):
    """Cached schedule for this input class (tuning on a miss when ``tune``)."""
    key = _class_of(x, metrics, precision, layout)
    hit = load_cache(path).get(key)
    if hit:
        return hit["schedule"]
    if not tune:
        return "auto"
    return tune_pairwise(x, metrics, precision, layout, path=path, **kw)[0]
