"""Python binding of the C ABI (same names), on PyTorch device tensors.

PyTorch supplies device memory and streams only; every step of the
computation runs in the library's CUDA kernels.  Metric requests are given as
strings or tuples:

    "l1" | "l2" | "gram" | ("lp", p)       -> root applied for distances
    ("l2", False) / ("lp", p, False)       -> raw integral int |f-g|^p

Functions raise ``PcfError`` on any non-OK status.  With ``check=True`` (the
default) a call synchronizes its stream and also raises for invalid PCF data
found on the device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import abi

__all__ = ["PcfError", "PcfTensors", "pcf_workspace_size", "pcf_prepare", "pcf_sort_order",
           "pcf_segment_integrals",
           "pcf_pairwise", "pcf_cross",
           "pcf_cross_to_host",
           "pcf_pairwise_backward", "pcf_check", "pcf_walk_promoted", "pcf_pairwise_weighted",
           "pcf_weighted_workspace_size", "pcf_cross_weighted", "PairwiseFn", "PairwiseGraph", "pdist",
           "l2_kernel", "pcf_reduce", "pcf_combine", "pcf_reduce_counters", "mean", "std",
           "parse_metric", "PRECISIONS", "REDUCTIONS", "OPS"]

PRECISIONS = {"f64": abi.PCF_PREC_F64, "f32c": abi.PCF_PREC_F32_COMP, "f32": abi.PCF_PREC_F32,
              "f32b": abi.PCF_PREC_F32_BLOCK,
              # float64 times rounded to float32 when packed (opt-in, faster)
              "f32c_round": abi.PCF_PREC_F32_COMP | abi.PCF_PREC_ROUND_TIMES,
              "f32_round": abi.PCF_PREC_F32 | abi.PCF_PREC_ROUND_TIMES,
              "f32b_round": abi.PCF_PREC_F32_BLOCK | abi.PCF_PREC_ROUND_TIMES,
              # float32 walk unless the input's dynamic range needs float64
              "f32c_auto64": abi.PCF_PREC_F32_COMP | abi.PCF_PREC_AUTO64,
              "f32_auto64": abi.PCF_PREC_F32 | abi.PCF_PREC_AUTO64,
              "f32b_auto64": abi.PCF_PREC_F32_BLOCK | abi.PCF_PREC_AUTO64}
REDUCTIONS = {"sum": abi.PCF_RED_SUM, "mean": abi.PCF_RED_MEAN, "max": abi.PCF_RED_MAX,
              "min": abi.PCF_RED_MIN, "std": abi.PCF_RED_STD}
OPS = {"add": abi.PCF_OP_ADD, "sub": abi.PCF_OP_SUB, "mul": abi.PCF_OP_MUL, "max": abi.PCF_OP_MAX,
       "min": abi.PCF_OP_MIN, "sqdiff": abi.PCF_OP_SQDIFF}
_METRICS = {"l1": abi.PCF_L1, "l2": abi.PCF_L2, "lp": abi.PCF_LP, "gram": abi.PCF_GRAM}


class PcfError(RuntimeError):
    def __init__(self, code, what, detail=None, index=None):
        msg = f"{what}: {abi.status_string(code)} (status {code})"
        if detail:
            msg += f"; {abi.ERR_DETAIL.get(detail, detail)} at index {index}"
        super().__init__(msg)
        self.code, self.detail, self.index = code, detail, index


@dataclass
class PcfTensors:
    """A CSR collection of PCFs on one CUDA device."""
    offsets: torch.Tensor   # int64 [N+1]
    times: torch.Tensor     # float32/float64 [nnz]
    values: torch.Tensor    # same dtype as times

    @property
    def n(self) -> int:
        return int(self.offsets.numel() - 1)

    @property
    def nnz(self) -> int:
        return int(self.times.numel())

    @staticmethod
    def from_numpy(s, device="cuda", dtype=None, pin=False):
        """Copy a host CSR set (anything with offsets/times/values) to `device`."""
        t, v = np.asarray(s.times), np.asarray(s.values)
        if dtype is not None:
            t, v = t.astype(dtype), v.astype(dtype)
        ts = [torch.from_numpy(np.ascontiguousarray(a)) for a in (s.offsets, t, v)]
        if pin:
            ts = [a.pin_memory() for a in ts]
        return PcfTensors(*(a.to(device, non_blocking=pin) for a in ts))

    def csr(self) -> abi.PcfCsr:
        for a in (self.offsets, self.times, self.values):
            if not a.is_cuda or not a.is_contiguous():
                raise ValueError("PcfTensors must be contiguous CUDA tensors")
        if self.offsets.dtype != torch.int64:
            raise ValueError("offsets must be int64")
        if self.times.dtype != self.values.dtype or self.times.dtype not in (torch.float32, torch.float64):
            raise ValueError("times/values must share float32 or float64")
        c = abi.PcfCsr()
        c.n, c.nnz = self.n, self.nnz
        c.offsets, c.times, c.values = (self.offsets.data_ptr(), self.times.data_ptr(),
                                        self.values.data_ptr())
        c.dtype = abi.PCF_F64 if self.times.dtype == torch.float64 else abi.PCF_F32
        return c


def parse_metric(m):
    """(metric_code, p, apply_root) from a request spec."""
    if isinstance(m, str):
        m = (m,)
    name = m[0].lower()
    if name not in _METRICS:
        raise ValueError(f"unknown metric {m!r}")
    code = _METRICS[name]
    if code == abi.PCF_LP:
        p = float(m[1])
        root = bool(m[2]) if len(m) > 2 else True
    else:
        p = {abi.PCF_L1: 1.0, abi.PCF_L2: 2.0, abi.PCF_GRAM: 1.0}[code]
        root = bool(m[1]) if len(m) > 1 else True
    return code, p, root


SCHEDULES = {"auto": abi.PCF_SCHED_AUTO, "tile1024": abi.PCF_SCHED_TILE_1024,
             "tile512x2": abi.PCF_SCHED_TILE_512X2, "tile512x3": abi.PCF_SCHED_TILE_512X3,
             "mergepath": abi.PCF_SCHED_MERGEPATH}


def _schedule(schedule, shard=None):
    """None | name | (name, window), plus an optional (shard_index,
    shard_count) -> PcfSchedule pointer or None."""
    if schedule is None and shard is None:
        return None
    if schedule is None:
        schedule = ("auto", 0)
    if isinstance(schedule, str):
        schedule = (schedule, 0)
    sc = abi.PcfSchedule()
    sc.kernel = SCHEDULES[schedule[0]]
    sc.window = int(schedule[1])
    if shard is not None:
        sc.shard_index, sc.shard_count = int(shard[0]), int(shard[1])
    return ctypes.byref(sc)


def _window(window):
    """None | (a, b) | (a, b, lam) -> PcfWindow pointer or None."""
    if window is None:
        return None
    w = abi.PcfWindow()
    w.a, w.b = float(window[0]), float(window[1])
    w.lam = float(window[2]) if len(window) > 2 else 0.0
    return ctypes.byref(w)


def _stream_handle(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _prec(precision):
    return PRECISIONS[precision] if isinstance(precision, str) else int(precision)


def pcf_workspace_size(x: PcfTensors, y: PcfTensors | None = None, precision="f32c",
                       purpose="forward") -> int:
    lib = abi.load()
    cx = x.csr()
    cy = y.csr() if y is not None else None
    out = ctypes.c_size_t(0)
    rc = lib.pcf_workspace_size(ctypes.byref(cx), ctypes.byref(cy) if cy else None,
                                _prec(precision),
                                abi.PCF_WS_BACKWARD if purpose == "backward" else abi.PCF_WS_FORWARD,
                                ctypes.byref(out))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_workspace_size")
    return int(out.value)


def _workspace(nbytes, device, workspace):
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError("workspace too small")
        return workspace
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def pcf_check(workspace: torch.Tensor, stream=None, what="pcf"):
    """Synchronize and raise if the device recorded invalid input."""
    lib = abi.load()
    detail = ctypes.c_int(0)
    index = ctypes.c_int64(-1)
    rc = lib.pcf_check(ctypes.c_void_p(workspace.data_ptr()), _stream_handle(stream),
                       ctypes.byref(detail), ctypes.byref(index))
    if rc != abi.PCF_OK:
        raise PcfError(rc, what, detail.value, index.value)


def pcf_walk_promoted(workspace: torch.Tensor, stream=None) -> bool:
    """True when the last PCF_PREC_AUTO64 call on `workspace` ran the float64
    walk (synchronizes)."""
    lib = abi.load()
    out = ctypes.c_int(0)
    rc = lib.pcf_walk_promoted(ctypes.c_void_p(workspace.data_ptr()), _stream_handle(stream),
                               ctypes.byref(out))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_walk_promoted")
    return bool(out.value)


def _requests(metrics, outs):
    arr = (abi.PcfIntegral * len(metrics))()
    for k, (m, o) in enumerate(zip(metrics, outs)):
        code, p, root = parse_metric(m)
        arr[k].metric, arr[k].p, arr[k].apply_root = code, p, int(root)
        arr[k].out = o.data_ptr() if o is not None and o.numel() else None
    return arr


def pcf_segment_integrals(x: PcfTensors, functional="lp", p=1.0, apply_root=False, a=0.0,
                          b=float("inf"), precision="f64", out_dtype=torch.float64, out=None,
                          workspace=None, stream=None, check=True):
    """Per-PCF integrals over [a, b] by segment iteration (Sec. 3.2, Alg. 3):
    ``"integral"`` gives int f dt, ``"lp"`` gives int |f|^p dt (the L_p norm
    with ``apply_root``).  Returns a length-N tensor."""
    lib = abi.load()
    fn = abi.PCF_FN_INTEGRAL if functional == "integral" else abi.PCF_FN_LP
    dev = x.times.device
    if out is None:
        out = torch.empty(x.n, dtype=out_dtype, device=dev)
    ws = _workspace(pcf_workspace_size(x, None, "f64"), dev, workspace)
    cx = x.csr()
    rc = lib.pcf_segment_integrals(ctypes.byref(cx), fn, float(p), int(bool(apply_root)),
                                   float(a), float(b), _prec(precision),
                                   ctypes.c_void_p(out.data_ptr()),
                                   abi.PCF_F64 if out.dtype == torch.float64 else abi.PCF_F32,
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                   _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_segment_integrals")
    if check:
        pcf_check(ws, stream, "pcf_segment_integrals")
    return out


def pcf_sort_order(x: PcfTensors, workspace: torch.Tensor, precision="f32c", stream=None):
    """perm (int32 device tensor): input index of the s-th PCF in the sort
    order of the collection prepared in ``workspace``."""
    lib = abi.load()
    perm = torch.empty(x.n, dtype=torch.int32, device=x.times.device)
    cx = x.csr()
    rc = lib.pcf_sort_order(ctypes.byref(cx), _prec(precision), ctypes.c_void_p(workspace.data_ptr()),
                            workspace.numel(), ctypes.c_void_p(perm.data_ptr()),
                            _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_sort_order")
    return perm


def pcf_prepare(x: PcfTensors, precision="f32c", workspace=None, stream=None):
    """Validate, sort and pack ``x`` into a workspace (returned) for later
    ``pcf_pairwise(..., prepared=True, workspace=ws)`` calls."""
    lib = abi.load()
    ws = _workspace(pcf_workspace_size(x, None, precision), x.times.device, workspace)
    cx = x.csr()
    rc = lib.pcf_prepare(ctypes.byref(cx), _prec(precision), ctypes.c_void_p(ws.data_ptr()),
                         ws.numel(), _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_prepare")
    return ws


def pcf_pairwise(x: PcfTensors, metrics=("l1",), precision="f32c", layout="full",
                 out_dtype=torch.float32, out=None, workspace=None, stream=None,
                 check=True, prepared=False, schedule=None, shard=None, window=None):
    """Pairwise matrices F(C) (Sec. 3.1) of ``x`` for each requested metric.

    ``window=(a, b)`` or ``(a, b, lam)`` integrates over [a, b] with the
    weight exp(-lam t) (tile schedules only).

    Returns a list of tensors: N x N (layout "full"), N(N+1)/2 ("upper"), or
    N x N in the library's sort order ("sorted"; see ``pcf_sort_order``)."""
    lib = abi.load()
    if isinstance(metrics, (str, tuple)):
        metrics = [metrics]
    metrics = list(metrics)
    n = x.n
    lay = {"full": abi.PCF_OUT_FULL, "upper": abi.PCF_OUT_UPPER_PACKED,
           "sorted": abi.PCF_OUT_FULL_SORTED}[layout]
    shape = (n * (n + 1) // 2,) if lay == abi.PCF_OUT_UPPER_PACKED else (n, n)
    dev = x.times.device
    if out is None:
        out = [torch.empty(shape, dtype=out_dtype, device=dev) for _ in metrics]
    ws = _workspace(pcf_workspace_size(x, None, precision), dev, workspace)
    cx = x.csr()
    req = _requests(metrics, out)
    od = abi.PCF_F64 if out[0].dtype == torch.float64 else abi.PCF_F32
    if prepared and workspace is None:
        raise ValueError("prepared=True needs the workspace returned by pcf_prepare")
    rc = lib.pcf_pairwise_ex(ctypes.byref(cx), req, len(metrics), _prec(precision), lay, od,
                             abi.PCF_PAIRWISE_PREPARED if prepared else 0,
                             _schedule(schedule, shard), _window(window),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_pairwise")
    if check:
        pcf_check(ws, stream, "pcf_pairwise")
    return out



def _weight_tensors(w, device):
    """A weight PCF as a one-PCF PcfTensors on `device`: PcfTensors, a host set
    with offsets/times/values, or a (times, values) pair."""
    if isinstance(w, PcfTensors):
        return w
    if hasattr(w, "offsets"):
        return PcfTensors.from_numpy(w, device)
    t, v = (np.asarray(a, dtype=np.float64) for a in w)
    o = np.array([0, t.size], dtype=np.int64)
    return PcfTensors(*(torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in (o, t, v)))


def pcf_weighted_workspace_size(x: PcfTensors, w, precision="f32c") -> int:
    lib = abi.load()
    cw = _weight_tensors(w, x.times.device).csr()
    cx = x.csr()
    out = ctypes.c_size_t()
    rc = lib.pcf_weighted_workspace_size(ctypes.byref(cx), ctypes.byref(cw), _prec(precision),
                                         ctypes.byref(out))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_weighted_workspace_size")
    return int(out.value)


def pcf_pairwise_weighted(x: PcfTensors, w, metrics=("l1",), precision="f32c", layout="full",
                          out_dtype=torch.float32, out=None, workspace=None, stream=None,
                          check=True, schedule=None):
    """Pairwise matrices r(int h(x_i, x_j) w dt) against one non-negative PCF
    weight ``w`` (weighted L_p of Sec. 2.2; weighted inner product for
    "gram"); layouts and precisions as ``pcf_pairwise``."""
    lib = abi.load()
    if isinstance(metrics, (str, tuple)):
        metrics = [metrics]
    metrics = list(metrics)
    n = x.n
    lay = {"full": abi.PCF_OUT_FULL, "upper": abi.PCF_OUT_UPPER_PACKED,
           "sorted": abi.PCF_OUT_FULL_SORTED}[layout]
    shape = (n * (n + 1) // 2,) if lay == abi.PCF_OUT_UPPER_PACKED else (n, n)
    dev = x.times.device
    wt = _weight_tensors(w, dev)
    if out is None:
        out = [torch.empty(shape, dtype=out_dtype, device=dev) for _ in metrics]
    ws = _workspace(pcf_weighted_workspace_size(x, wt, precision), dev, workspace)
    cx, cw = x.csr(), wt.csr()
    req = _requests(metrics, out)
    od = abi.PCF_F64 if out[0].dtype == torch.float64 else abi.PCF_F32
    rc = lib.pcf_pairwise_weighted(ctypes.byref(cx), ctypes.byref(cw), req, len(metrics),
                                   _prec(precision), lay, od, _schedule(schedule),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                   _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_pairwise_weighted")
    if check:
        pcf_check(ws, stream, "pcf_pairwise_weighted")
    return out


def pcf_cross_weighted(a: PcfTensors, b: PcfTensors, w, row_begin=0, row_end=None,
                       metrics=("l1",), precision="f32c", out_dtype=torch.float32, out=None,
                       ld_out=None, workspace=None, stream=None, check=True, schedule=None):
    """Cross block r(int h(a_i, b_j) w dt) for rows [row_begin, row_end) of
    ``a`` against all of ``b``, for one non-negative PCF weight ``w``."""
    lib = abi.load()
    if isinstance(metrics, (str, tuple)):
        metrics = [metrics]
    metrics = list(metrics)
    row_end = a.n if row_end is None else row_end
    rows = row_end - row_begin
    dev = b.times.device
    wt = _weight_tensors(w, dev)
    ld = b.n if ld_out is None else ld_out
    if out is None:
        out = [torch.empty((rows, ld), dtype=out_dtype, device=dev) for _ in metrics]
    ca, cb, cw = a.csr(), b.csr(), wt.csr()
    size = ctypes.c_size_t()
    rc = lib.pcf_cross_weighted_workspace_size(ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(cw),
                                               _prec(precision), ctypes.byref(size))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_cross_weighted_workspace_size")
    ws = _workspace(int(size.value), dev, workspace)
    req = _requests(metrics, out)
    od = abi.PCF_F64 if out[0].dtype == torch.float64 else abi.PCF_F32
    rc = lib.pcf_cross_weighted(ctypes.byref(ca), ctypes.byref(cb), row_begin, row_end,
                                ctypes.byref(cw), req, len(metrics), _prec(precision), ld, od,
                                _schedule(schedule), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_cross_weighted")
    if check:
        pcf_check(ws, stream, "pcf_cross_weighted")
    return out

def pcf_cross(a: PcfTensors, b: PcfTensors, row_begin=0, row_end=None, metrics=("l1",),
              precision="f32c", out_dtype=torch.float32, out=None, ld_out=None,
              reuse_b=False, workspace=None, stream=None, check=True, schedule=None,
              shard=None, window=None):
    """Rows [row_begin, row_end) of the cross matrices a x b."""
    lib = abi.load()
    if isinstance(metrics, (str, tuple)):
        metrics = [metrics]
    metrics = list(metrics)
    row_end = a.n if row_end is None else row_end
    rows = row_end - row_begin
    ld = b.n if ld_out is None else ld_out
    dev = b.times.device
    if out is None:
        out = [torch.empty((rows, ld), dtype=out_dtype, device=dev) for _ in metrics]
    ws = _workspace(pcf_workspace_size(a, b, precision), dev, workspace)
    ca, cb = a.csr(), b.csr()
    req = _requests(metrics, out)
    od = abi.PCF_F64 if out[0].dtype == torch.float64 else abi.PCF_F32
    rc = lib.pcf_cross_ex(ctypes.byref(ca), ctypes.byref(cb), int(row_begin), int(row_end), req,
                          len(metrics), _prec(precision), int(ld), od,
                          abi.PCF_CROSS_REUSE_B if reuse_b else 0, _schedule(schedule, shard),
                          _window(window),
                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_cross")
    if check:
        pcf_check(ws, stream, "pcf_cross")
    return out


def pcf_pairwise_backward(x: PcfTensors, metric, grad_out: torch.Tensor, fwd_out=None,
                          workspace=None, stream=None, check=True, shard=None):
    """(grad_values, grad_times) of sum(grad_out * F) for the FULL matrix F.
    ``shard=(rank, world)``: this GPU's share (tiles t with t % world == rank);
    the shares sum to the whole gradient."""
    lib = abi.load()
    code, p, root = parse_metric(metric)
    dev = x.times.device
    gv = torch.empty_like(x.values)
    gt = torch.empty_like(x.times)
    ws = _workspace(pcf_workspace_size(x, None, "f64", "backward"), dev, workspace)
    g = grad_out.contiguous()
    if g.dtype not in (torch.float32, torch.float64):
        g = g.to(torch.float64)
    f = None
    if fwd_out is not None:
        f = fwd_out.contiguous()
        if f.dtype != g.dtype:
            raise ValueError("fwd_out and grad_out must share a dtype")
    cx = x.csr()
    rc = lib.pcf_pairwise_backward_ex(
        ctypes.byref(cx), code, p, int(root),
        ctypes.c_void_p(f.data_ptr()) if f is not None else None,
        ctypes.c_void_p(g.data_ptr()), abi.PCF_F64 if g.dtype == torch.float64 else abi.PCF_F32,
        ctypes.c_void_p(gv.data_ptr()), ctypes.c_void_p(gt.data_ptr()),
        _schedule(None, shard), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_pairwise_backward")
    if check:
        pcf_check(ws, stream, "pcf_pairwise_backward")
    return gv, gt


def pcf_pairwise_to_host(x: PcfTensors, metrics=("l1",), precision="f32c",
                         out_dtype=torch.float32, host_out=None, out=None, bands=0,
                         workspace=None, stream=None, copy_stream=None, check=True,
                         schedule=None):
    """FULL pairwise matrices (as ``pcf_pairwise``) streamed to page-locked
    host memory while they are computed: the walk runs in bands, and the rows
    a band completes are copied to ``host_out`` on ``copy_stream`` while the
    next band runs.  ``out``: the device matrices (allocated if None);
    ``bands``: 0 = the library's default.  Returns the host tensors."""
    lib = abi.load()
    if isinstance(metrics, (str, tuple)):
        metrics = [metrics]
    metrics = list(metrics)
    n = x.n
    dev = x.times.device
    if out is None:
        out = [torch.empty((n, n), dtype=out_dtype, device=dev) for _ in metrics]
    if host_out is None:
        host_out = [torch.empty((n, n), dtype=out[0].dtype).pin_memory() for _ in metrics]
    for h, o in zip(host_out, out):
        if not h.is_pinned() or h.dtype != o.dtype or h.numel() != n * n or not h.is_contiguous():
            raise ValueError("host_out: contiguous page-locked N x N tensors of the output dtype")
    ws = _workspace(pcf_workspace_size(x, None, precision), dev, workspace)
    cx = x.csr()
    req = _requests(metrics, out)
    od = abi.PCF_F64 if out[0].dtype == torch.float64 else abi.PCF_F32
    ptrs = (ctypes.c_void_p * len(metrics))(*[h.data_ptr() for h in host_out])
    if copy_stream is None:
        copy_stream = torch.cuda.Stream(dev)
    rc = lib.pcf_pairwise_to_host(ctypes.byref(cx), req, len(metrics), _prec(precision), od,
                                  _schedule(schedule), ptrs, int(bands),
                                  ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  _stream_handle(stream), ctypes.c_void_p(copy_stream.cuda_stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_pairwise_to_host")
    if check:
        pcf_check(ws, stream, "pcf_pairwise_to_host")
    return host_out


def pcf_cross_to_host(a: PcfTensors, b: PcfTensors, metrics=("l1",), precision="f32c",
                      block_rows=2048, out_dtype=torch.float32, host_out=None, schedule=None,
                      check=True):
    """Cross matrices a x b streamed to pinned host memory block by block.

    Row blocks of ``a`` are computed with ``pcf_cross`` into two alternating
    device buffers; while block k+1 is computed, block k is copied to the
    host on a separate stream (b is validated and packed once, then reused).
    Returns the host tensors (``a.n`` x ``b.n`` per metric)."""
    if isinstance(metrics, (str, tuple)):
        metrics = [metrics]
    metrics = list(metrics)
    dev = b.times.device
    na, nb = a.n, b.n
    if host_out is None:
        host_out = [torch.empty((na, nb), dtype=out_dtype).pin_memory() for _ in metrics]
    if na == 0 or nb == 0:
        return host_out
    rows = max(1, min(block_rows, na))
    bufs = [[torch.empty((rows, nb), dtype=out_dtype, device=dev) for _ in metrics]
            for _ in range(2)]
    ws = torch.empty(max(pcf_workspace_size(a, b, precision), 256), dtype=torch.uint8, device=dev)
    compute = torch.cuda.current_stream(dev)
    copy = torch.cuda.Stream(dev)
    freed = [None, None]
    for k, r0 in enumerate(range(0, na, rows)):
        r1 = min(na, r0 + rows)
        slot = k % 2
        if freed[slot] is not None:
            compute.wait_event(freed[slot])
        views = [t[: r1 - r0] for t in bufs[slot]]
        pcf_cross(a, b, r0, r1, metrics, precision=precision, out=views, workspace=ws,
                  reuse_b=k > 0, check=False, schedule=schedule)
        done = torch.cuda.Event()
        done.record(compute)
        copy.wait_event(done)
        with torch.cuda.stream(copy):
            for h, v in zip(host_out, views):
                h[r0:r1].copy_(v, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(copy)
        freed[slot] = ev
    compute.wait_stream(copy)
    if check:
        pcf_check(ws, what="pcf_cross_to_host")
        copy.synchronize()
    return host_out


class PairwiseFn(torch.autograd.Function):
    """F = pairwise matrix of one metric, differentiable in values and times.

    The backward pass recomputes the merge walks (nothing but the output F is
    saved)."""

    @staticmethod
    def forward(ctx, values, times, offsets, metric="l2", precision="f64"):
        x = PcfTensors(offsets, times.detach(), values.detach())
        out_dtype = values.dtype
        F = pcf_pairwise(x, [metric], precision=precision, out_dtype=out_dtype)[0]
        ctx.save_for_backward(values, times, offsets, F)
        ctx.metric = metric
        return F

    @staticmethod
    def backward(ctx, grad):
        values, times, offsets, F = ctx.saved_tensors
        x = PcfTensors(offsets, times.detach(), values.detach())
        gv, gt = pcf_pairwise_backward(x, ctx.metric, grad.to(F.dtype), fwd_out=F)
        return gv, gt, None, None, None


class PairwiseGraph:
    """pcf_prepare + pcf_pairwise captured once into a CUDA graph and replayed.

    For repeated calls on collections of the same shape (same N and nnz,
    new contents copied into ``x``'s tensors): the validation, sort, pack and
    walk launches are replayed as one graph, with the workspace and outputs
    allocated once.  ``replay()`` enqueues on the current stream; call
    ``check()`` to synchronize and surface invalid input."""

    def __init__(self, x: PcfTensors, metrics, precision="f32c", layout="full",
                 out_dtype=torch.float32, schedule=None):
        self.x = x
        self.metrics = list(metrics) if not isinstance(metrics, (str, tuple)) else [metrics]
        n = x.n
        shape = (n * (n + 1) // 2,) if layout == "upper" else (n, n)
        self.outs = [torch.empty(shape, dtype=out_dtype, device=x.times.device)
                     for _ in self.metrics]
        self.ws = torch.empty(max(pcf_workspace_size(x, None, precision), 256),
                              dtype=torch.uint8, device=x.times.device)
        args = dict(precision=precision, layout=layout, out=self.outs, workspace=self.ws,
                    check=False, schedule=schedule)
        # run once outside capture (module loading, kernel attributes)
        pcf_prepare(x, precision, workspace=self.ws)
        pcf_pairwise(x, self.metrics, prepared=True, **args)
        pcf_check(self.ws)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            pcf_prepare(x, precision, workspace=self.ws)
            pcf_pairwise(x, self.metrics, prepared=True, **args)

    def replay(self):
        self.graph.replay()
        return self.outs

    def check(self):
        pcf_check(self.ws, what="PairwiseGraph")


def pdist(x: PcfTensors, p=1.0, precision="f64", out_dtype=torch.float64):
    """L_p distance matrix (the paper's ``pdist``, Sec. 5.2)."""
    return pcf_pairwise(x, [("lp", p)], precision=precision, out_dtype=out_dtype)[0]


def l2_kernel(x: PcfTensors, precision="f64", out_dtype=torch.float64):
    """L2 inner-product (Gram) matrix (the paper's ``l2_kernel``, Sec. 5.2)."""
    return pcf_pairwise(x, ["gram"], precision=precision, out_dtype=out_dtype)[0]


# Short names of the two matrix calls (pairwise matrix of one collection,
# cross matrix of two; Sec. 3.1)
pairwise = pcf_pairwise
cross = pcf_cross


def _csr_out(n_out, capacity, device):
    off = torch.empty(n_out + 1, dtype=torch.int64, device=device)
    t = torch.empty(max(capacity, 1), dtype=torch.float64, device=device)
    v = torch.empty(max(capacity, 1), dtype=torch.float64, device=device)
    c = abi.PcfCsrOut()
    c.capacity, c.offsets, c.times, c.values = capacity, off.data_ptr(), t.data_ptr(), v.data_ptr()
    return c, off, t, v


def _trimmed(off, t, v):
    rows = int(off[-1].item())
    return PcfTensors(off, t[:rows], v[:rows])


def pcf_reduce_workspace_size(x: PcfTensors, group_size, reduction="mean", std_rows=0) -> int:
    lib = abi.load()
    out = ctypes.c_size_t(0)
    cx = x.csr()
    rc = lib.pcf_reduce_workspace_size(ctypes.byref(cx), int(group_size), REDUCTIONS[reduction],
                                       int(std_rows), ctypes.byref(out))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_reduce_workspace_size")
    return int(out.value)


def pcf_reduce_counters(workspace: torch.Tensor, stream=None):
    """(merge positions, rows written) of the last reduction on ``workspace``."""
    lib = abi.load()
    pos, rows = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib.pcf_reduce_counters(ctypes.c_void_p(workspace.data_ptr()), _stream_handle(stream),
                                 ctypes.byref(pos), ctypes.byref(rows))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_reduce_counters")
    return int(pos.value), int(rows.value)


def pcf_reduce(x: PcfTensors, group_size=None, reduction="mean", workspace=None, stream=None,
               check=True, trim=True, out=None):
    """Reduce each run of ``group_size`` consecutive PCFs (default: all of x)
    to one PCF by a binary tree of ReducePair nodes (Sec. 4, Alg. 4, Fig. 2):
    ``"sum"``, ``"mean"``, ``"max"``, ``"min"`` or the sample ``"std"``
    (Sec. 2.1, factor 1/(m - 1)).  Returns float64 PcfTensors with one PCF
    per group.  With ``trim`` the call synchronizes to size the result."""
    lib = abi.load()
    m = x.n if group_size is None else int(group_size)
    if m < 1 or x.n % m:
        raise ValueError("group_size must divide the number of PCFs")
    dev = x.times.device
    if workspace is None:
        std_rows = 0
        if reduction == "std":
            # exact intermediate size from the means: nnz + m * rows of the means
            std_rows = x.nnz + m * pcf_reduce(x, m, "mean", stream=stream, check=check).nnz
        ws = _workspace(pcf_reduce_workspace_size(x, m, reduction, std_rows), dev, None)
    else:
        ws = workspace      # its capacity is checked by the library
    if out is None:
        out = _csr_out(x.n // m, x.nnz, dev)
    out, off, t, v = out
    cx = x.csr()
    rc = lib.pcf_reduce(ctypes.byref(cx), m, REDUCTIONS[reduction], ctypes.byref(out),
                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_reduce")
    if check:
        pcf_check(ws, stream, "pcf_reduce")
    return _trimmed(off, t, v) if trim else PcfTensors(off, t, v)


def pcf_combine(a: PcfTensors, b: PcfTensors, op="add", workspace=None, stream=None, check=True,
                trim=True):
    """Elementwise h_*(a_i, b_i) (b with a's count) or h_*(a_i, b_0) (b with
    one PCF) by ReducePair (Sec. 4, Alg. 4), h one of ``OPS``."""
    lib = abi.load()
    ca, cb = a.csr(), b.csr()
    nbytes = ctypes.c_size_t(0)
    rc = lib.pcf_combine_workspace_size(ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(nbytes))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_combine_workspace_size")
    dev = a.times.device
    ws = _workspace(int(nbytes.value), dev, workspace)
    cap = a.nnz + b.nnz if b.n == a.n else a.nnz + a.n * b.nnz
    out, off, t, v = _csr_out(a.n, cap, dev)
    rc = lib.pcf_combine(ctypes.byref(ca), ctypes.byref(cb), OPS[op], ctypes.byref(out),
                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream))
    if rc != abi.PCF_OK:
        raise PcfError(rc, "pcf_combine")
    if check:
        pcf_check(ws, stream, "pcf_combine")
    return _trimmed(off, t, v) if trim else PcfTensors(off, t, v)


def mean(x: PcfTensors, group_size=None, **kw):
    """Mean of each group of PCFs (the paper's ``mean``, Sec. 5.1)."""
    return pcf_reduce(x, group_size, "mean", **kw)


def std(x: PcfTensors, group_size=None, **kw):
    """Sample standard deviation of each group of PCFs (Sec. 2.1)."""
    return pcf_reduce(x, group_size, "std", **kw)
