"""The C-ABI library loads without a GPU, exports every symbol the header
declares, agrees with the generator on the weights-blob size, rejects invalid
descriptors, and reports a clean error (no crash) when no device is present."""

import ctypes
import os
import re

import numpy as np
import pytest

from synth import configs, weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2104_04547_gb300 import build
    build.build()
    from paper_2104_04547_gb300 import fusion
    return fusion


def _declared():
    src = open(os.path.join(ROOT, "include", "fusion.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fusion_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(F):
    lib = ctypes.CDLL(F.LIB_PATH)
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), n


def test_blob_size_matches_generator(F):
    for name in configs.MODELS:
        d = configs.model(name)
        assert F.fusion_weights_bytes(F.make_desc(d)) == weights.blob_size(d)


def test_invalid_descriptors_give_zero_bytes(F):
    d = configs.model("fusion-24grid-c32")
    for field, val in (("grid_n", 2), ("support", 9), ("sg_hidden", 48)):
        bad = dict(d)
        bad[field] = val
        assert F.fusion_weights_bytes(F.make_desc(bad)) == 0
    bad = configs.model("fusion-24grid-c32")
    bad["head"] = [64, 2]
    assert F.fusion_weights_bytes(F.make_desc(bad)) == 0
    assert "last head layer" in F.fusion_last_error()


def test_create_without_device_is_an_error_not_a_crash(F):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    d = configs.model("fusion-24grid-c32")
    blob = weights.to_blob(d, weights.init_weights(d, 0))
    with pytest.raises(F.FusionError) as e:
        F.fusion_create(F.make_desc(d, max_poses=1), blob)
    assert e.value.code in (F.FUSION_ECUDA, F.FUSION_ENOMEM)


def test_best_per_compound_matches_numpy_groupby(F):
    """The per-compound maximum over poses (no device needed): values and the first index reaching them."""
    rng = np.random.default_rng(5)
    n, nc = 500, 37
    comp = rng.integers(0, nc - 2, n).astype(np.int32)           # compounds nc-2, nc-1 have no poses
    aff = np.round(rng.standard_normal(n).astype(np.float32), 1)   # rounding makes ties
    best, idx = F.fusion_best_per_compound(aff, comp, nc)
    for c in range(nc):
        sel = np.nonzero(comp == c)[0]
        if len(sel) == 0:
            assert best[c] == -np.inf and idx[c] == -1
            continue
        m = aff[sel].max()
        assert best[c] == m and idx[c] == sel[np.argmax(aff[sel] == m)]


def test_best_per_compound_rejects_bad_input(F):
    with pytest.raises(F.FusionError):
        F.fusion_best_per_compound(np.zeros(3, np.float32), np.array([0, 1, 5], np.int32), 3)
    with pytest.raises(F.FusionError):
        F.fusion_best_per_compound(np.array([0, np.nan, 1], np.float32), np.zeros(3, np.int32), 1)
