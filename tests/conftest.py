"""Shared pytest configuration: the `gpu` marker and golden-file helpers."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


def read_golden(name):
    """Parse a golden file into {section_header: [row, ...]} with float rows."""
    sections = {}
    cur = None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                sections[cur] = []
                continue
            sections[cur].append([float(x) for x in line.split()])
    return {k: np.array(v, dtype=np.float64) for k, v in sections.items()}


@pytest.fixture(scope="session")
def golden():
    return read_golden


def max_rel_error(metric, got, want, gram_diag=None):
    """Per-matrix error measure: distances max |x - x*| / |x*| (x* = 0 only
    where both are exactly 0); Gram |x - x*| / sqrt(G*_ii G*_jj)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    both_inf = np.isinf(got) & np.isinf(want) & (np.sign(got) == np.sign(want))
    diff = np.abs(got - want)
    diff[both_inf] = 0.0
    if metric == "gram":
        d = np.sqrt(np.abs(np.asarray(gram_diag, dtype=np.float64)))
        scale = np.outer(d, d) if want.ndim == 2 else d
        scale = np.where(scale > 0, scale, 1.0)
    else:
        scale = np.abs(want)
        zero = scale == 0
        if np.any(diff[zero] != 0):
            return np.inf
        scale = np.where(zero, 1.0, scale)
    r = diff / scale
    r[both_inf] = 0.0
    if np.any(np.isnan(got) != np.isnan(want)):
        return np.inf
    return float(np.nanmax(r)) if r.size else 0.0


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
