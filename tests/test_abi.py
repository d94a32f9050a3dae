"""The C-ABI library loads without a GPU, exports every symbol the header
declares, agrees with the generator on the weights-blob size, rejects invalid
descriptors (each rule of the descriptor check broken alone, with its own
message), and reports a clean error (no crash) when no device is present."""

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


def test_binding_constants_match_the_header(F):
    src = open(os.path.join(ROOT, "include", "fusion.h")).read()
    defs = dict(re.findall(r"#define\s+(FUSION_(?:OPT|STAGE)_[A-Z0-9_]+)\s+(-?\d+)", src))
    assert len([k for k in defs if k.startswith("FUSION_OPT_")]) >= 7
    for name, value in defs.items():
        py = name if name.startswith("FUSION_OPT_") else name[len("FUSION_"):]   # stages: F.STAGE_*
        assert getattr(F, py, None) == int(value), name


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


def _conv(i, **kw):
    def f(d):
        for k, v in kw.items():
            setattr(d.conv[i], k, v)
    return f


def _set(**kw):
    def f(d):
        for k, v in kw.items():
            setattr(d, k, v)
    return f


# (what breaks, change to a valid small-model descriptor, fragment of the error message)
BAD_DESCRIPTORS = [
    ("feature count", _set(n_feat=18), "n_feat must be 19"),
    ("grid side", _set(grid_n=97), "grid_n must be in [4, 96]"),
    ("voxel size zero", _set(grid_h=0.0), "grid_h must be > 0"),
    ("voxel size NaN", _set(grid_h=float("nan")), "grid_h must be > 0"),
    ("Gaussian width", _set(sigma=-1.0), "sigma must be > 0"),
    ("support", _set(support=0), "support must be in [1, 5]"),
    ("no conv layers", _set(n_conv=0), "n_conv must be in [1, 8]"),
    ("first conv input channels", _conv(0, c_in=20), "conv c_in must equal"),
    ("conv output channels", _conv(0, c_out=48), "conv c_out must be a multiple of 32"),
    ("even kernel", _conv(0, k=4), "conv k must be odd"),
    ("stride 3", _conv(1, stride=3, residual=0), "conv stride must be 1 or 2"),
    ("strided residual", _conv(1, stride=2), "residual conv needs c_in == c_out and stride 1"),
    ("pool", _set(pool=3), "pool must be 0, 1 or 2"),
    ("CNN dense width", _set(cnn_dense=0), "cnn_dense must be in [1, 512]"),
    ("graph stages", _set(sg_n_stages=3), "sg_n_stages must be 1 or 2"),
    ("graph steps", lambda d: d.sg_steps.__setitem__(0, 17), "sg_steps must be in [0, 16]"),
    ("empty edge mask", lambda d: d.sg_edges.__setitem__(0, 0), "sg_edges must be a non-empty"),
    ("stage gate flag", _set(sg_gate=2), "sg_gate must be 0 or 1"),
    ("gather kind", _set(sg_gather=5), "bad sg_gather"),
    ("gather width", _set(sg_gather_width=0), "sg_gather_width must be in [1, 256]"),
    ("latent width", _set(cnn_dense=400, sg_gather_width=200), "CNN latent width + sg_gather_width must be <= 512"),
    ("second CNN dense width", _set(cnn_dense2=513), "cnn_dense2 must be in [0, 512]"),
    ("first CNN dense width with a second", _set(cnn_dense=60, cnn_dense2=32), "cnn_dense must be a multiple of 8"),
    ("latent width with a second CNN dense", _set(cnn_dense2=500, sg_gather_width=64),
     "CNN latent width + sg_gather_width must be <= 512"),
    ("stage width above the hidden width", lambda d: d.sg_width.__setitem__(0, 40),
     "sg_width must be 0 or in [1, sg_hidden]"),
    ("first stage narrower than the features", lambda d: d.sg_width.__setitem__(0, 18),
     "the first stage's width must hold the 19 features"),
    ("unequal stage widths without a gate",
     lambda d: (_set(sg_n_stages=2, sg_gate=0)(d), d.sg_steps.__setitem__(1, 1), d.sg_edges.__setitem__(1, 3),
                d.sg_width.__setitem__(0, 19), d.sg_width.__setitem__(1, 24)),
     "stages of unequal widths need sg_gate"),
    ("fusion form", _set(fusion=7), "bad fusion form"),
    ("branch layers on coherent fusion", lambda d: (_set(n_cnn_out=1)(d), d.cnn_out.__setitem__(0, 32)),
     "coherent fusion has no branch layers"),
    ("cutoffs out of order", _set(cut_nc=1.0), "cutoffs must satisfy 0 < cut_cov < cut_nc"),
    ("no fusion layers", _set(n_head=0), "n_head must be in [1, 6]"),
    ("dtype", _set(dtype=9), "bad dtype"),
    ("pose capacity", _set(max_poses=0), "max_poses must be in [1, 65535]"),
    ("atom capacity", _set(max_atoms=4097), "max_atoms must be in [1, 4096]"),
    ("degree capacity", _set(max_degree=0), "max_degree must be in [1, 1024]"),
]


@pytest.mark.parametrize("what,change,msg", BAD_DESCRIPTORS, ids=[b[0] for b in BAD_DESCRIPTORS])
def test_each_descriptor_rule_rejects_its_violation(F, what, change, msg):
    """Every check of the model descriptor, broken alone on a valid descriptor, gives 0 bytes and its message."""
    good = F.make_desc(configs.model("fusion-24grid-c32"), max_poses=4)
    assert F.fusion_weights_bytes(good) > 0
    bad = F.make_desc(configs.model("fusion-24grid-c32"), max_poses=4)
    change(bad)
    assert F.fusion_weights_bytes(bad) == 0, what
    assert msg in F.fusion_last_error(), (what, F.fusion_last_error())


def test_mid_and_late_fusion_rules(F):
    mid = F.make_desc(configs.model("fusion-24grid-c32-mid"))
    assert F.fusion_weights_bytes(mid) > 0
    mid.n_sg_out = 0
    assert F.fusion_weights_bytes(mid) == 0 and "mid and late fusion need branch layers" in F.fusion_last_error()
    late = F.make_desc(configs.model("fusion-24grid-c32-late"))
    assert F.fusion_weights_bytes(late) > 0
    late.cnn_out[late.n_cnn_out - 1] = 2
    assert F.fusion_weights_bytes(late) == 0 and "must end in width 1" in F.fusion_last_error()
    late = F.make_desc(configs.model("fusion-24grid-c32-late"))
    late.n_head = 1
    late.head[0] = 1
    assert F.fusion_weights_bytes(late) == 0 and "late fusion has no fusion layers" in F.fusion_last_error()
