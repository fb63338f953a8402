import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def read_golden(name):
    """Parse a tests/golden/*.txt file: '<key> v1 v2 ...' lines, '#' comments."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(v) for v in vals]
    return out


def elem_rel(got, want):
    """Largest error of any element relative to that element's largest value (floored at
    1e-3 of the global largest value): a handful of wrong nodes fails it even where the
    2-norm over a whole array would not notice them.  Arrays shaped [..., K, 4, Np]."""
    import numpy as np
    g = np.asarray(got, dtype=np.float64)
    w = np.asarray(want, dtype=np.float64)
    K = w.shape[-3]
    err = np.abs(g - w).reshape(-1, K, w.shape[-2] * w.shape[-1]).max(axis=(0, 2))
    scale = np.abs(w).reshape(-1, K, w.shape[-2] * w.shape[-1]).max(axis=(0, 2))
    scale = np.maximum(scale, 1e-3 * scale.max())
    return float((err / scale).max())
