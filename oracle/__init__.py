"""CPU oracle for the PCF integral matrices -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

Two independent implementations of the same definition,

    F_ij = r( int_0^inf h(f_i(t), f_j(t)) dt )          (Sec. 2.2, Sec. 3.1)

evaluated as the sum over the common refinement of the two breakpoint sets of
h(f(s_k), g(s_k)) (s_{k+1} - s_k)                       (Sec. 3, Eq. simpleint):

* ``pcf_oracle.c`` (loaded through ctypes): float64 rectangle iteration
  (Alg. 1) with accumulation (Alg. 2), threaded over matrix rows, plus the
  adjoint (gradient of sum G * F with respect to values and times).
  It also holds the reductions of Sec. 4: ReducePair (Alg. 4) and binary
  reduction trees (Fig. 2) for sums, means, maxima, minima and the sample
  standard deviation of Sec. 2.1.
* ``brute.py``: the common refinement built explicitly (sort + unique), values
  looked up by binary search, summed with numpy; and an exact rational
  version for tiny inputs.

``build()`` compiles the C file with the system C compiler into
``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lib = None
_lock = threading.Lock()

METRICS = {"l1": 0, "l2": 1, "lp": 2, "gram": 3}

OPS = {"add": 0, "sub": 1, "mul": 2, "max": 3, "min": 4, "sqdiff": 5}
REDUCTIONS = {"sum": 0, "mean": 1, "max": 2, "min": 3, "std": 4}

__all__ = ["build", "integral", "integral_ab", "rectangles", "matrix", "backward", "segment_integral",
           "merge_steps", "total_merge_steps", "segment_sq", "reduce_pair", "reduce", "METRICS",
           "OPS", "REDUCTIONS"]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no fast-math) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dbl, ip = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            P = ctypes.c_void_p
            lib.orc_integral.restype = dbl
            lib.orc_integral.argtypes = [P, P, i64, P, P, i64, ip, dbl]
            lib.orc_rectangles.restype = i64
            lib.orc_rectangles.argtypes = [P, P, i64, P, P, i64, P, P, P, P, i64]
            lib.orc_merge_steps.restype = i64
            lib.orc_merge_steps.argtypes = [P, i64, P, i64]
            lib.orc_matrix.restype = None
            lib.orc_matrix.argtypes = [i64, P, P, P, i64, P, P, P, i64, i64,
                                       ip, dbl, ip, P, ip]
            lib.orc_segment_sq.restype = dbl
            lib.orc_segment_sq.argtypes = [P, P, i64]
            lib.orc_integral_ab.restype = dbl
            lib.orc_integral_ab.argtypes = [P, P, i64, P, P, i64, ip, dbl, dbl, dbl, dbl]
            lib.orc_integral_w.restype = dbl
            lib.orc_integral_w.argtypes = [P, P, i64, P, P, i64, P, P, i64, ip, dbl]
            lib.orc_segment_integral.restype = dbl
            lib.orc_segment_integral.argtypes = [P, P, i64, ip, dbl, dbl, dbl]
            lib.orc_reduce_pair.restype = i64
            lib.orc_reduce_pair.argtypes = [P, P, i64, P, P, i64, ip, P, P]
            lib.orc_reduce.restype = i64
            lib.orc_reduce.argtypes = [i64, i64, P, P, P, ip, P, P, P, i64, ip]
            lib.orc_backward.restype = None
            lib.orc_backward.argtypes = [i64, P, P, P, ip, dbl, ip, P, P, P]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _metric(m):
    return METRICS[m] if isinstance(m, str) else int(m)


def integral(tf, vf, tg, vg, metric="l1", p=1.0) -> float:
    """int_0^inf h(f, g) dt for one pair (no root)."""
    tf, vf, tg, vg = map(_f64, (tf, vf, tg, vg))
    return _load().orc_integral(_ptr(tf), _ptr(vf), tf.size, _ptr(tg), _ptr(vg),
                                tg.size, _metric(metric), float(p))


def integral_ab(tf, vf, tg, vg, metric="l1", p=1.0, a=0.0, b=float("inf"), lam=0.0) -> float:
    """int_a^b h(f, g) exp(-lam t) dt (no root)."""
    tf, vf, tg, vg = map(_f64, (tf, vf, tg, vg))
    return _load().orc_integral_ab(_ptr(tf), _ptr(vf), tf.size, _ptr(tg), _ptr(vg), tg.size,
                                   _metric(metric), float(p), float(a), float(b), float(lam))


def integral_w(tf, vf, tg, vg, tw, vw, metric="l1", p=1.0) -> float:
    """int_0^inf h(f, g) w dt for a non-negative PCF weight w (no root)."""
    tf, vf, tg, vg, tw, vw = map(_f64, (tf, vf, tg, vg, tw, vw))
    return _load().orc_integral_w(_ptr(tf), _ptr(vf), tf.size, _ptr(tg), _ptr(vg), tg.size,
                                  _ptr(tw), _ptr(vw), tw.size, _metric(metric), float(p))


def matrix_w(a, w, b=None, metric="l1", p=1.0, apply_root=True) -> np.ndarray:
    """Weighted pairwise (b None) or cross matrix: r(int h(a_i, b_j) w dt)
    with w = (times, values) one PCF; pair by pair (small inputs)."""
    bb = a if b is None else b
    tw, vw = _f64(w[0]), _f64(w[1])
    out = np.empty((a.n, bb.n))
    for i in range(a.n):
        tf, vf = a.pcf(i)
        for j in range(bb.n):
            if b is None and j < i:
                out[i, j] = out[j, i]
                continue
            I = integral_w(tf, vf, *bb.pcf(j), tw, vw, metric, p)
            out[i, j] = _root(metric, p, I) if apply_root else I
    return out


def _root(metric, p, x):
    if metric == "gram":
        return x
    e = {"l1": 1.0, "l2": 2.0}.get(metric, p)
    if e == 1.0:
        return x
    if e == 2.0:
        return float(np.sqrt(x))
    return x ** (1.0 / e)


def rectangles(tf, vf, tg, vg):
    """The rectangles (l, r, v_f, v_g) of Alg. 1 over [0, inf), as an (m, 4) array."""
    tf, vf, tg, vg = map(_f64, (tf, vf, tg, vg))
    cap = tf.size + tg.size + 2
    out = [np.empty(cap) for _ in range(4)]
    m = _load().orc_rectangles(_ptr(tf), _ptr(vf), tf.size, _ptr(tg), _ptr(vg),
                               tg.size, *[_ptr(o) for o in out], cap)
    return np.stack([o[:m] for o in out], axis=1)


def merge_steps(tf, tg) -> int:
    """|T_f u T_g|: the number of rectangles of the pair, tail included."""
    tf, tg = _f64(tf), _f64(tg)
    return int(_load().orc_merge_steps(_ptr(tf), tf.size, _ptr(tg), tg.size))


def total_merge_steps(a, b=None, pairs=None) -> int:
    """Sum of |T_f u T_g| over the upper triangle (with diagonal) of set ``a``,
    over all of ``a`` x ``b``, or over an explicit (k, 2) index array."""
    lib = _load()
    ta = _f64(a.times)
    oa = a.offsets
    if b is None and pairs is None:
        pairs = [(i, j) for i in range(a.n) for j in range(i, a.n)]
        tb, ob = ta, oa
    elif pairs is None:
        tb, ob = _f64(b.times), b.offsets
        pairs = [(i, j) for i in range(a.n) for j in range(b.n)]
    else:
        tb, ob = (ta, oa) if b is None else (_f64(b.times), b.offsets)
    s = 0
    base_a = ta.ctypes.data
    base_b = tb.ctypes.data
    for i, j in pairs:
        s += lib.orc_merge_steps(ctypes.c_void_p(base_a + 8 * int(oa[i])),
                                 int(oa[i + 1] - oa[i]),
                                 ctypes.c_void_p(base_b + 8 * int(ob[j])),
                                 int(ob[j + 1] - ob[j]))
    return s


def matrix(a, b=None, metric="l1", p=1.0, apply_root=True, rows=None,
           nthreads=None) -> np.ndarray:
    """F(C) for the pairwise matrix of ``a`` (``b`` None) or the cross matrix
    ``a`` x ``b``; ``rows`` = (begin, end) restricts to a block of rows."""
    lib = _load()
    ta, va = _f64(a.times), _f64(a.values)
    oa = np.ascontiguousarray(a.offsets, dtype=np.int64)
    r0, r1 = (0, a.n) if rows is None else (int(rows[0]), int(rows[1]))
    if b is None:
        ncol = a.n
        args_b = (0, None, None, None)
    else:
        tb, vb = _f64(b.times), _f64(b.values)
        ob = np.ascontiguousarray(b.offsets, dtype=np.int64)
        ncol = b.n
        args_b = (b.n, _ptr(ob), _ptr(tb), _ptr(vb))
    out = np.empty((r1 - r0, ncol))
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib.orc_matrix(a.n, _ptr(oa), _ptr(ta), _ptr(va), *args_b, r0, r1,
                   _metric(metric), float(p), int(bool(apply_root)), _ptr(out),
                   int(nthreads))
    return out


def segment_sq(t, v) -> float:
    """int_0^inf f^2 dt by segment iteration (Alg. 3)."""
    t, v = _f64(t), _f64(v)
    return _load().orc_segment_sq(_ptr(t), _ptr(v), t.size)


def segment_integral(t, v, kind="lp", p=1.0, a=0.0, b=float("inf")) -> float:
    """int_a^b h(f) dt by segment iteration (Alg. 3); kind "integral" uses
    h(v) = v, kind "lp" uses |v|^p (no root)."""
    t, v = _f64(t), _f64(v)
    return _load().orc_segment_integral(_ptr(t), _ptr(v), t.size, 0 if kind == "integral" else 1,
                                        float(p), float(a), float(b))


def backward(a, G, metric="l2", p=2.0, apply_root=False):
    """(grad_values, grad_times) of sum_ij G_ij F_ij, both shaped like a.values."""
    lib = _load()
    ta, va = _f64(a.times), _f64(a.values)
    oa = np.ascontiguousarray(a.offsets, dtype=np.int64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    gv = np.empty(a.nnz)
    gt = np.empty(a.nnz)
    lib.orc_backward(a.n, _ptr(oa), _ptr(ta), _ptr(va), _metric(metric),
                     float(p), int(bool(apply_root)), _ptr(G), _ptr(gv), _ptr(gt))
    return gv, gt


def reduce_pair(tf, vf, tg, vg, op="add"):
    """ReducePair (Alg. 4): breakpoints and values of h_*(f, g)."""
    tf, vf, tg, vg = map(_f64, (tf, vf, tg, vg))
    out_t = np.empty(tf.size + tg.size)
    out_v = np.empty(tf.size + tg.size)
    n = _load().orc_reduce_pair(_ptr(tf), _ptr(vf), tf.size, _ptr(tg), _ptr(vg), tg.size,
                                OPS[op], _ptr(out_t), _ptr(out_v))
    return out_t[:n].copy(), out_v[:n].copy()


def reduce(a, group_size, red="mean", nthreads=None):
    """Reduce consecutive groups of ``group_size`` PCFs of ``a`` (a.n must be a
    multiple) to one PCF each: (offsets, times, values) as numpy arrays."""
    lib = _load()
    m = int(group_size)
    if m < 1 or a.n % m:
        raise ValueError("group_size must divide the number of PCFs")
    groups = a.n // m
    ta, va = _f64(a.times), _f64(a.values)
    oa = np.ascontiguousarray(a.offsets, dtype=np.int64)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    cap = max(int(a.nnz), 1)
    while True:
        out_off = np.empty(groups + 1, dtype=np.int64)
        out_t, out_v = np.empty(cap), np.empty(cap)
        n = lib.orc_reduce(groups, m, _ptr(oa), _ptr(ta), _ptr(va), REDUCTIONS[red],
                           _ptr(out_off), _ptr(out_t), _ptr(out_v), cap, int(nthreads))
        if n >= 0:
            return out_off, out_t[:n].copy(), out_v[:n].copy()
        cap = int(out_off[-1])
