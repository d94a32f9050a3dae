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


# ---- a conv layer in isolation: the GPU's own input map (fetched), convolved in float64 on the CPU ----

def _torch():
    return pytest.importorskip("torch")


def to_bf16(a):
    """Round to bf16 (nearest even) and back to float64."""
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def to_e4m3(a):
    """Round to FP8 E4M3 (nearest even, saturating at 448) and back to float64."""
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()


def check_layer_bf16(x_in, W, b, cv, y_gpu):
    """x_in: [n][n][n][C] float (exact bf16 values), weights rounded to bf16; y_gpu: [m][m][m][Co].  Within
    the output's bf16 rounding plus FP32 accumulation."""
    from oracle import fusion_oracle as O
    x = np.asarray(x_in, dtype=np.float64)
    ref = np.maximum(O.conv3d(x, to_bf16(W), b.astype(np.float64), cv["stride"]), 0.0)
    if cv["residual"]:
        ref = ref + x
    scale = float(np.abs(ref).max()) + 1e-12
    err = np.abs(y_gpu - ref)
    assert np.all(err <= 8e-3 * np.abs(ref) + 2e-3 * scale), (float(err.max()), scale)


def check_layer_fp8(x_bf16, W, b, cv, y_gpu):
    """Input quantized per pose (max |x| / 448), weights per output channel, both E4M3, as the FP8 path does;
    within 2e-2 of the output's largest magnitude (E4M3 codes computed on the host may differ from the GPU's
    by one step where a value sits on a rounding boundary)."""
    from oracle import fusion_oracle as O
    x = np.asarray(x_bf16, dtype=np.float64)
    s_in = np.abs(x).max() / 448.0
    xq = to_e4m3(x / s_in) * s_in
    co = W.shape[0]
    sw = np.abs(W.reshape(co, -1)).max(axis=1) / 448.0
    wq = to_e4m3(W / sw[:, None, None, None, None]) * sw[:, None, None, None, None]
    ref = np.maximum(O.conv3d(xq, wq, b.astype(np.float64), cv["stride"]), 0.0)
    if cv["residual"]:
        ref = ref + x
    scale = float(np.abs(ref).max()) + 1e-12
    err = float(np.abs(y_gpu - ref).max())
    assert err <= 2e-2 * scale, (err, scale)


def layers_in_isolation(F, m, desc, W, p, check, layers=None):
    """Check conv layers of pose p of the last call one by one against `check` (needs keep_stages)."""
    n = desc["grid_n"]
    x = m.fetch(F.STAGE_GRID, p).reshape(n, n, n, 19)
    for i, cv in enumerate(desc["conv"]):
        y = m.fetch(F.STAGE_CONV, (i << 16) | p)
        side = round((y.size // cv["c_out"]) ** (1 / 3))
        y = y.reshape(side, side, side, cv["c_out"])
        if layers is None or i in layers:
            check(x, W[f"conv{i}.w"], W[f"conv{i}.b"], cv, y)
        x = y
