"""Helpers shared by the GPU parity tests."""

from __future__ import annotations

import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

# FP32 path tolerance on the affinity (absolute), as the method's target states.
F32_AFFINITY_TOL = 1e-4


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_04547_gb300 import build
    build.build()
    from paper_2104_04547_gb300 import fusion
    return fusion


def golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


def local_csr(rp, col):
    return np.asarray(rp, dtype=np.int64), np.asarray(col, dtype=np.int64)


def split_csr(buf, n):
    rp = buf[:n + 1]
    col = buf[n + 1:]
    return rp, col
