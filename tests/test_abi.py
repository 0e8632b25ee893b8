"""Host-side checks of the C ABI library (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2404_07183_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "pcf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pcf_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load()


def test_header_declares_the_abi():
    decl = _declared_functions()
    assert set(decl) == set(abi.SYMBOLS), decl


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert lib.pcf_version().decode().startswith("pcf_gb300")
    assert lib.pcf_status_string(abi.PCF_ENOWS).decode().startswith("workspace")


def _csr(n, nnz, dtype=abi.PCF_F32):
    c = abi.PcfCsr()
    c.n, c.nnz, c.dtype = n, nnz, dtype
    c.offsets = c.times = c.values = 0x1000 if n else 0
    return c


def test_workspace_size_host_only(lib):
    out = ctypes.c_size_t()
    x = _csr(1000, 55000)
    assert lib.pcf_workspace_size(ctypes.byref(x), None, abi.PCF_PREC_F32_COMP,
                                  abi.PCF_WS_FORWARD, ctypes.byref(out)) == abi.PCF_OK
    f32 = out.value
    assert f32 >= 55000 * 8 + 1000 * 4 * 5 + 1001 * 8
    assert lib.pcf_workspace_size(ctypes.byref(x), None, abi.PCF_PREC_F64,
                                  abi.PCF_WS_FORWARD, ctypes.byref(out)) == abi.PCF_OK
    assert out.value >= f32 + 55000 * 8
    assert lib.pcf_workspace_size(ctypes.byref(x), None, abi.PCF_PREC_F64,
                                  abi.PCF_WS_BACKWARD, ctypes.byref(out)) == abi.PCF_OK
    assert out.value >= 55000 * (16 + 16)
    y = _csr(10, 100)
    assert lib.pcf_workspace_size(ctypes.byref(x), ctypes.byref(y), abi.PCF_PREC_F32,
                                  abi.PCF_WS_FORWARD, ctypes.byref(out)) == abi.PCF_OK
    bad = _csr(-1, 0)
    assert lib.pcf_workspace_size(ctypes.byref(bad), None, abi.PCF_PREC_F32,
                                  abi.PCF_WS_FORWARD, ctypes.byref(out)) == abi.PCF_EINVAL
    assert lib.pcf_workspace_size(ctypes.byref(x), None, 7, abi.PCF_WS_FORWARD,
                                  ctypes.byref(out)) == abi.PCF_EINVAL


def test_workspace_size_of_the_precision_modifiers(lib):
    """float64 input in a float32 precision packs 16-byte keyed elements plus
    the key sort's buffers; the rounded-times opt-in packs 8-byte elements;
    AUTO64 holds either form; both modifiers are invalid with PCF_PREC_F64."""
    out = ctypes.c_size_t()

    def size(x, prec):
        rc = lib.pcf_workspace_size(ctypes.byref(x), None, prec, abi.PCF_WS_FORWARD,
                                    ctypes.byref(out))
        return out.value if rc == abi.PCF_OK else rc

    x64, x32 = _csr(1000, 55000, abi.PCF_F64), _csr(1000, 55000, abi.PCF_F32)
    keyed = size(x64, abi.PCF_PREC_F32_COMP)
    rounded = size(x64, abi.PCF_PREC_F32_COMP | abi.PCF_PREC_ROUND_TIMES)
    assert rounded == size(x32, abi.PCF_PREC_F32_COMP)
    assert keyed >= rounded + 55000 * (8 + 2 * 8 + 2 * 4)
    assert size(x64, abi.PCF_PREC_F32_COMP | abi.PCF_PREC_AUTO64) >= keyed
    assert size(x32, abi.PCF_PREC_F32_COMP | abi.PCF_PREC_AUTO64) >= size(x32, abi.PCF_PREC_F64)
    for mod in (abi.PCF_PREC_ROUND_TIMES, abi.PCF_PREC_AUTO64, 0x400):
        assert size(x64, abi.PCF_PREC_F64 | mod) == abi.PCF_EINVAL


def test_argument_errors_return_before_any_device_work(lib):
    x = _csr(10, 100)
    req = (abi.PcfIntegral * 1)()
    req[0].metric, req[0].p, req[0].out = abi.PCF_L1, 1.0, 0x2000
    s = ctypes.c_void_p(0)
    assert lib.pcf_pairwise(None, req, 1, 0, 0, 0, 0, None, 0, s) == abi.PCF_EINVAL
    assert lib.pcf_pairwise(ctypes.byref(x), req, 0, 0, 0, 0, 0, None, 0, s) == abi.PCF_EINVAL
    assert lib.pcf_pairwise(ctypes.byref(x), req, 1, 9, 0, 0, 0, None, 0, s) == abi.PCF_EINVAL
    assert lib.pcf_pairwise(ctypes.byref(x), req, 1, 0, 5, 0, 0, None, 0, s) == abi.PCF_EINVAL
    req[0].metric, req[0].p = abi.PCF_LP, 0.5
    assert lib.pcf_pairwise(ctypes.byref(x), req, 1, 0, 0, 0, 0, None, 0, s) == abi.PCF_EINVAL
    req[0].metric, req[0].p = abi.PCF_L1, 1.0
    # workspace missing / misaligned / too small
    assert lib.pcf_pairwise(ctypes.byref(x), req, 1, 0, 0, 0, 0, None, 1 << 20, s) == abi.PCF_ENOWS
    assert lib.pcf_pairwise(ctypes.byref(x), req, 1, 0, 0, 0, 0, ctypes.c_void_p(0x1008),
                            1 << 20, s) == abi.PCF_ENOWS
    assert lib.pcf_pairwise(ctypes.byref(x), req, 1, 0, 0, 0, 0, ctypes.c_void_p(0x1000),
                            16, s) == abi.PCF_ENOWS
    a, b = _csr(10, 100), _csr(5, 50)
    assert lib.pcf_cross(ctypes.byref(a), ctypes.byref(b), 3, 2, req, 1, 0, 5, 0, 0,
                         None, 0, s) == abi.PCF_EINVAL
    assert lib.pcf_cross(ctypes.byref(a), ctypes.byref(b), 0, 10, req, 1, 0, 4, 0, 0,
                         None, 0, s) == abi.PCF_EINVAL
    assert lib.pcf_pairwise_backward(ctypes.byref(x), 9, 1.0, 0, None, None, 1, None, None,
                                     None, 0, s) == abi.PCF_EINVAL
    # root with exponent != 1 needs the forward output
    assert lib.pcf_pairwise_backward(ctypes.byref(x), abi.PCF_L2, 2.0, 1, None,
                                     ctypes.c_void_p(0x1000), 1, ctypes.c_void_p(0x1000),
                                     ctypes.c_void_p(0x1000), None, 0, s) == abi.PCF_EINVAL


def test_to_host_argument_errors_return_before_any_device_work(lib):
    x = _csr(10, 100)
    req = (abi.PcfIntegral * 1)()
    req[0].metric, req[0].p, req[0].out = abi.PCF_L1, 1.0, 0x2000
    host = (ctypes.c_void_p * 1)(0x3000)
    s = ctypes.c_void_p(0)
    ws, wsb = ctypes.c_void_p(0x1000), 1 << 20
    f = lib.pcf_pairwise_to_host
    assert f(None, req, 1, 1, 0, None, host, 0, ws, wsb, s, s) == abi.PCF_EINVAL
    assert f(ctypes.byref(x), req, 1, 9, 0, None, host, 0, ws, wsb, s, s) == abi.PCF_EINVAL
    assert f(ctypes.byref(x), req, 1, 1, 5, None, host, 0, ws, wsb, s, s) == abi.PCF_EINVAL
    assert f(ctypes.byref(x), req, 1, 1, 0, None, host, -1, ws, wsb, s, s) == abi.PCF_EINVAL
    assert f(ctypes.byref(x), req, 0, 1, 0, None, host, 0, ws, wsb, s, s) == abi.PCF_EINVAL
    sched = abi.PcfSchedule()
    sched.shard_index, sched.shard_count = 0, 2      # no shards when streaming
    assert f(ctypes.byref(x), req, 1, 1, 0, ctypes.byref(sched), host, 0, ws, wsb, s,
             s) == abi.PCF_EINVAL
    assert f(ctypes.byref(x), req, 1, 1, 0, None, host, 0, None, wsb, s, s) == abi.PCF_ENOWS
    assert f(ctypes.byref(x), req, 1, 1, 0, None, None, 0, ws, wsb, s, s) == abi.PCF_EINVAL
    empty = _csr(0, 0)
    assert f(ctypes.byref(empty), req, 1, 1, 0, None, None, 0, ws, wsb, s, s) == abi.PCF_OK


def test_empty_collection_is_a_no_op(lib):
    x = _csr(0, 0)
    req = (abi.PcfIntegral * 1)()
    req[0].metric = abi.PCF_GRAM
    assert lib.pcf_pairwise(ctypes.byref(x), req, 1, 0, 0, 0, 0, ctypes.c_void_p(0x1000),
                            1 << 20, ctypes.c_void_p(0)) == abi.PCF_OK


def test_product_package_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2404_07183_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "pcf_oracle" not in text and "liborc" not in text, f
