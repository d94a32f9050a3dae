"""ctypes binding of the C ABI in ``include/fusion.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls; all scoring
work runs in the CUDA library ``libfusion_gb300.so``.  Importing this module
fails loudly when the library has not been built: there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfusion_gb300.so")

FUSION_OK = 0
FUSION_EINVAL = -1
FUSION_EWEIGHTS = -2
FUSION_ENOMEM = -3
FUSION_ECAPACITY = -4
FUSION_ECUDA = -5
FUSION_ETIMEOUT = -6
FUSION_EUNSUPPORTED = -7
FUSION_EAGAIN = -8

FUSION_F32, FUSION_BF16, FUSION_FP8 = 0, 1, 2
DTYPES = {"f32": FUSION_F32, "bf16": FUSION_BF16, "fp8": FUSION_FP8}

MAX_CONV, MAX_STAGES, MAX_HEAD = 8, 2, 6

STAGE_ORIGIN, STAGE_GRID, STAGE_CONV, STAGE_POOL, STAGE_CNN_LATENT = 1, 2, 3, 4, 5
STAGE_EDGES_COV, STAGE_EDGES_NC, STAGE_SG_STATE, STAGE_SG_LATENT, STAGE_AFFINITY = 6, 7, 8, 9, 10

TIMING_NAMES = ["prep", "voxelize"] + [f"conv{i}" for i in range(8)] + \
               ["maxpool", "cnn_dense", "radius_graph", "sg_steps", "sg_gather", "head", "total"]

FUSION_COHERENT, FUSION_MID, FUSION_LATE = 0, 1, 2
FUSION_FORMS = {"coherent": FUSION_COHERENT, "mid": FUSION_MID, "late": FUSION_LATE}

FUSION_OPT_CUDA_GRAPH = 1
FUSION_OPT_CONV_SLICES_PER_MMA = 2
FUSION_OPT_TEST_WAIT_TIMEOUT = 3
FUSION_OPT_GRAPH_NODES_PER_WARP = 4
FUSION_OPT_SERIAL_BRANCHES = 5
FUSION_OPT_GRAPH_TENSOR_CORES = 6
FUSION_OPT_CONV_STRIDE2_SPLIT = 7

EXPORTED = ["fusion_weights_bytes", "fusion_create", "fusion_score", "fusion_destroy", "fusion_last_error",
            "fusion_stage_bytes", "fusion_fetch_stage", "fusion_last_timings", "fusion_cnn_dense_noalloc",
            "fusion_server_create", "fusion_server_submit", "fusion_server_submit_dtype", "fusion_server_poll", "fusion_server_drain",
            "fusion_server_get_stats", "fusion_server_destroy", "fusion_set_option", "fusion_autotune",
            "fusion_describe_conv", "fusion_best_per_compound", "fusion_graph_schedule"]

FUSION_NOALLOC_MAX_PARTIALS = 1 << 21


class FusionError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fusion error {code}: {msg}")
        self.code = code


class fusion_conv_desc(C.Structure):
    _fields_ = [("c_in", C.c_int32), ("c_out", C.c_int32), ("k", C.c_int32), ("stride", C.c_int32),
                ("residual", C.c_int32)]


class fusion_model_desc(C.Structure):
    _fields_ = [("n_feat", C.c_int32), ("grid_n", C.c_int32), ("grid_h", C.c_float), ("sigma", C.c_float),
                ("support", C.c_int32), ("n_conv", C.c_int32), ("conv", fusion_conv_desc * MAX_CONV),
                ("pool", C.c_int32), ("cnn_dense", C.c_int32), ("sg_hidden", C.c_int32),
                ("sg_n_stages", C.c_int32), ("sg_steps", C.c_int32 * MAX_STAGES),
                ("sg_edges", C.c_int32 * MAX_STAGES), ("sg_gate", C.c_int32), ("sg_gather", C.c_int32),
                ("sg_gather_width", C.c_int32), ("cut_cov", C.c_float), ("cut_nc", C.c_float),
                ("n_head", C.c_int32), ("head", C.c_int32 * MAX_HEAD), ("dtype", C.c_int32),
                ("max_poses", C.c_int32), ("max_atoms", C.c_int32), ("max_degree", C.c_int32),
                ("keep_stages", C.c_int32), ("fusion", C.c_int32), ("n_cnn_out", C.c_int32),
                ("cnn_out", C.c_int32 * MAX_HEAD), ("n_sg_out", C.c_int32), ("sg_out", C.c_int32 * MAX_HEAD),
                ("head_residual", C.c_int32), ("cnn_dense2", C.c_int32), ("sg_width", C.c_int32 * MAX_STAGES)]


class fusion_poses(C.Structure):
    _fields_ = [("n_poses", C.c_int32), ("atom_off", C.c_void_p), ("n_lig", C.c_void_p), ("xyz", C.c_void_p),
                ("feat", C.c_void_p), ("on_device", C.c_int32)]


class fusion_server_config(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("batch_window_us", C.c_double),
                ("hbm_budget_bytes", C.c_size_t), ("queue_capacity", C.c_int32), ("dtypes", C.c_int32)]


class fusion_server_stats(C.Structure):
    _fields_ = [("slots", C.c_int32), ("slot_bytes", C.c_size_t), ("submitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("failed", C.c_int64), ("batches", C.c_int64), ("queued", C.c_int64),
                ("inflight", C.c_int64), ("gpu_busy_s", C.c_double), ("slots_by_dtype", C.c_int32 * 3)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built ({LIB_PATH}); run paper_2104_04547_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    lib.fusion_weights_bytes.argtypes = [P(fusion_model_desc)]
    lib.fusion_weights_bytes.restype = C.c_size_t
    lib.fusion_create.argtypes = [P(fusion_model_desc), C.c_void_p, C.c_size_t, C.c_void_p, P(C.c_void_p)]
    lib.fusion_create.restype = C.c_int
    lib.fusion_score.argtypes = [C.c_void_p, P(fusion_poses), C.c_int32, C.c_void_p]
    lib.fusion_score.restype = C.c_int
    lib.fusion_destroy.argtypes = [C.c_void_p]
    lib.fusion_destroy.restype = None
    lib.fusion_last_error.argtypes = []
    lib.fusion_last_error.restype = C.c_char_p
    lib.fusion_stage_bytes.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    lib.fusion_stage_bytes.restype = C.c_int64
    lib.fusion_fetch_stage.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t]
    lib.fusion_fetch_stage.restype = C.c_int
    lib.fusion_last_timings.argtypes = [C.c_void_p, P(C.c_float), C.c_int32]
    lib.fusion_last_timings.restype = C.c_int
    lib.fusion_cnn_dense_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                             C.c_int32, C.c_void_p, C.c_void_p]
    lib.fusion_cnn_dense_noalloc.restype = C.c_int
    lib.fusion_server_create.argtypes = [P(fusion_model_desc), C.c_void_p, C.c_size_t, P(fusion_server_config),
                                         P(C.c_void_p)]
    lib.fusion_server_create.restype = C.c_int
    lib.fusion_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, P(C.c_uint64)]
    lib.fusion_server_submit.restype = C.c_int
    lib.fusion_server_submit_dtype.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                               P(C.c_uint64)]
    lib.fusion_server_submit_dtype.restype = C.c_int
    lib.fusion_server_poll.argtypes = [C.c_void_p, C.c_uint64, P(C.c_float), P(C.c_double)]
    lib.fusion_server_poll.restype = C.c_int
    lib.fusion_server_drain.argtypes = [C.c_void_p, C.c_double]
    lib.fusion_server_drain.restype = C.c_int
    lib.fusion_server_get_stats.argtypes = [C.c_void_p, P(fusion_server_stats)]
    lib.fusion_server_get_stats.restype = C.c_int
    lib.fusion_server_destroy.argtypes = [C.c_void_p]
    lib.fusion_server_destroy.restype = None
    lib.fusion_set_option.argtypes = [C.c_void_p, C.c_int32, C.c_int64]
    lib.fusion_set_option.restype = C.c_int
    lib.fusion_autotune.argtypes = [C.c_void_p, P(fusion_poses), C.c_int32]
    lib.fusion_autotune.restype = C.c_int
    lib.fusion_describe_conv.argtypes = [C.c_void_p, C.c_int32, P(C.c_int32)]
    lib.fusion_describe_conv.restype = C.c_int
    lib.fusion_best_per_compound.argtypes = [P(C.c_float), P(C.c_int32), C.c_int32, C.c_int32, P(C.c_float),
                                             P(C.c_int32)]
    lib.fusion_best_per_compound.restype = C.c_int
    lib.fusion_graph_schedule.argtypes = [C.c_void_p, P(C.c_int32)]
    lib.fusion_graph_schedule.restype = C.c_int
    return lib


lib = _load()


def fusion_last_error() -> str:
    return lib.fusion_last_error().decode()


def _check(rc):
    if rc != FUSION_OK:
        raise FusionError(rc, fusion_last_error())


def make_desc(model: dict, max_poses: int = 64, max_atoms: int = 1200, max_degree: int = 64,
              keep_stages: bool = False, dtype: str | None = None) -> fusion_model_desc:
    """C descriptor from a model dict (see ``synth.configs``)."""
    d = fusion_model_desc()
    d.n_feat = model["n_feat"]
    d.grid_n = model["grid_n"]
    d.grid_h = model["grid_h"]
    d.sigma = model["sigma"]
    d.support = model["support"]
    d.n_conv = len(model["conv"])
    for i, cv in enumerate(model["conv"]):
        d.conv[i] = fusion_conv_desc(cv["c_in"], cv["c_out"], cv["k"], cv["stride"], cv["residual"])
    d.pool = model["pool"]
    d.cnn_dense = model["cnn_dense"]
    d.sg_hidden = model["sg_hidden"]
    d.sg_n_stages = len(model["sg_stages"])
    for s, st in enumerate(model["sg_stages"]):
        d.sg_steps[s] = st["steps"]
        d.sg_edges[s] = st["edges"]
    d.sg_gate = model["sg_gate"]
    d.sg_gather = 1 if model["sg_gather"] == "gated" else 0
    d.sg_gather_width = model["sg_gather_width"]
    d.cut_cov = model["cut_cov"]
    d.cut_nc = model["cut_nc"]
    d.n_head = len(model["head"])
    for l, w in enumerate(model["head"]):
        d.head[l] = w
    d.fusion = FUSION_FORMS[model.get("fusion", "coherent")]
    d.n_cnn_out = len(model.get("cnn_out", []))
    for l, w in enumerate(model.get("cnn_out", [])):
        d.cnn_out[l] = w
    d.n_sg_out = len(model.get("sg_out", []))
    for l, w in enumerate(model.get("sg_out", [])):
        d.sg_out[l] = w
    d.head_residual = int(model.get("head_residual", 0))
    d.cnn_dense2 = int(model.get("cnn_dense2", 0))
    for s, w in enumerate(model.get("sg_width", []) or []):
        d.sg_width[s] = int(w)
    d.dtype = DTYPES[dtype or model["dtype"]]
    d.max_poses = max_poses
    d.max_atoms = max_atoms
    d.max_degree = max_degree
    d.keep_stages = int(keep_stages)
    return d


def fusion_weights_bytes(desc: fusion_model_desc) -> int:
    return int(lib.fusion_weights_bytes(C.byref(desc)))


def fusion_create(desc: fusion_model_desc, weights, stream=None) -> C.c_void_p:
    """weights: bytes or a host buffer; stream: cudaStream_t as an int (None: library-owned stream)."""
    buf = weights if isinstance(weights, (bytes, bytearray)) else np.ascontiguousarray(weights).tobytes()
    h = C.c_void_p()
    cbuf = C.create_string_buffer(bytes(buf), len(buf)) if len(buf) else None
    rc = lib.fusion_create(C.byref(desc), cbuf, len(buf), C.c_void_p(stream) if stream else None, C.byref(h))
    _check(rc)
    return h


def fusion_destroy(model) -> None:
    lib.fusion_destroy(model)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _poses_struct(poses, n_poses, on_device, keep):
    if not on_device:
        arrs = {
            "atom_off": np.ascontiguousarray(poses["atom_off"], dtype=np.int32),
            "n_lig": np.ascontiguousarray(poses["n_lig"], dtype=np.int32),
            "xyz": np.ascontiguousarray(poses["xyz"], dtype=np.float32),
            "feat": np.ascontiguousarray(poses["feat"], dtype=np.float32),
        }
        keep.append(arrs)
        src = arrs
    else:
        src = poses
    return fusion_poses(n_poses, _ptr(src["atom_off"]), _ptr(src["n_lig"]), _ptr(src["xyz"]), _ptr(src["feat"]),
                        int(on_device))


def fusion_set_option(model, option: int, value: int) -> None:
    _check(lib.fusion_set_option(model, option, value))


def fusion_autotune(model, poses: dict, n_poses: int, on_device: bool = False) -> None:
    keep = []
    P = _poses_struct(poses, n_poses, on_device, keep)
    _check(lib.fusion_autotune(model, C.byref(P), n_poses))


def fusion_best_per_compound(affinity, compound, n_compounds: int):
    """Strongest affinity of each compound over its poses and the first pose reaching it
    (-inf and -1 for a compound without poses)."""
    aff = np.ascontiguousarray(affinity, dtype=np.float32)
    cmp_ = np.ascontiguousarray(compound, dtype=np.int32)
    if aff.shape != cmp_.shape:
        raise ValueError("affinity and compound differ in length")
    best = np.empty(n_compounds, dtype=np.float32)
    idx = np.empty(n_compounds, dtype=np.int32)
    P = C.POINTER
    _check(lib.fusion_best_per_compound(aff.ctypes.data_as(P(C.c_float)), cmp_.ctypes.data_as(P(C.c_int32)),
                                        len(aff), n_compounds, best.ctypes.data_as(P(C.c_float)),
                                        idx.ctypes.data_as(P(C.c_int32))))
    return best, idx


def fusion_describe_conv(model, layer: int) -> dict:
    out = (C.c_int32 * 5)()
    _check(lib.fusion_describe_conv(model, layer, out))
    return {"slices_per_cta": out[0], "groups_per_stage": out[1], "stages": out[2], "smem_bytes": out[3],
            "slices_per_mma": out[4]}


def fusion_graph_schedule(model) -> int:
    npw = C.c_int32(0)
    _check(lib.fusion_graph_schedule(model, C.byref(npw)))
    return int(npw.value)


def fusion_score(model, poses: dict, n_poses: int, out, on_device: bool = False) -> None:
    """Score a packed batch.

    poses: dict with atom_off, n_lig, xyz, feat as host numpy arrays (on_device
    False) or device buffers (torch CUDA tensors or raw int pointers, on_device
    True).  out: float32 [n_poses] host array or device buffer, matching.
    """
    keep = []
    if not on_device:
        arrs = {
            "atom_off": np.ascontiguousarray(poses["atom_off"], dtype=np.int32),
            "n_lig": np.ascontiguousarray(poses["n_lig"], dtype=np.int32),
            "xyz": np.ascontiguousarray(poses["xyz"], dtype=np.float32),
            "feat": np.ascontiguousarray(poses["feat"], dtype=np.float32),
        }
        keep.append(arrs)
        src = arrs
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float32 and out.flags.c_contiguous
    else:
        src = poses
    P = fusion_poses(n_poses, _ptr(src["atom_off"]), _ptr(src["n_lig"]), _ptr(src["xyz"]), _ptr(src["feat"]),
                     int(on_device))
    rc = lib.fusion_score(model, C.byref(P), n_poses, C.c_void_p(_ptr(out)))
    _check(rc)


def fusion_stage_bytes(model, stage: int, index: int) -> int:
    n = int(lib.fusion_stage_bytes(model, stage, index))
    if n < 0:
        _check(n)
    return n


def fusion_fetch_stage(model, stage: int, index: int = 0) -> np.ndarray:
    """Intermediate result of the last scoring call as a numpy array (float32 or int32)."""
    n = fusion_stage_bytes(model, stage, index)
    dt = np.int32 if stage in (STAGE_EDGES_COV, STAGE_EDGES_NC) else np.float32
    out = np.empty(n // 4, dtype=dt)
    _check(lib.fusion_fetch_stage(model, stage, index, out.ctypes.data, n))
    return out


def fusion_last_timings(model, n: int = 17) -> np.ndarray:
    out = (C.c_float * n)()
    _check(lib.fusion_last_timings(model, out, n))
    return np.array(out[:], dtype=np.float32)


def fusion_cnn_dense_noalloc(x, w, bias, B: int, N: int, K: int, relu: bool, y, stream=None) -> None:
    """Dense layer with the library's fixed scratch (no allocation); device buffers in and out."""
    rc = lib.fusion_cnn_dense_noalloc(C.c_void_p(_ptr(x)), C.c_void_p(_ptr(w)), C.c_void_p(_ptr(bias)), B, N, K,
                                      int(relu), C.c_void_p(_ptr(y)), C.c_void_p(stream) if stream else None)
    _check(rc)


class Model:
    """Owns a model handle: ``Model(model_dict, weights_blob, max_poses=...)``."""

    def __init__(self, model: dict, weights, max_poses=64, max_atoms=1200, max_degree=64,
                 keep_stages=False, stream=None, dtype=None):
        self.spec = model
        self.desc = make_desc(model, max_poses, max_atoms, max_degree, keep_stages, dtype)
        self.handle = fusion_create(self.desc, weights, stream)

    def score(self, poses, n_poses=None, out=None, on_device=False):
        if n_poses is None:
            n_poses = len(poses["n_lig"])
        if out is None:
            out = np.empty(n_poses, dtype=np.float32)
        fusion_score(self.handle, poses, n_poses, out, on_device)
        return out

    def fetch(self, stage, index=0):
        return fusion_fetch_stage(self.handle, stage, index)

    def timings(self):
        return dict(zip(TIMING_NAMES, fusion_last_timings(self.handle).tolist()))

    def use_cuda_graphs(self, on=True):
        fusion_set_option(self.handle, FUSION_OPT_CUDA_GRAPH, int(on))

    def serial_branches(self, on=True):
        """Measurement mode: both branches on one stream, so timings() gives each stage's own kernel time."""
        fusion_set_option(self.handle, FUSION_OPT_SERIAL_BRANCHES, int(on))

    def graph_tensor_cores(self, on=-1):
        """1: graph steps' GRU and transforms on the tensor cores (three-term BF16 split); 0: FP32 CUDA
        cores; -1: the dtype's default (tensor cores for BF16 / FP8)."""
        fusion_set_option(self.handle, FUSION_OPT_GRAPH_TENSOR_CORES, int(on))

    def conv_stride2_split(self, on=-1):
        """1 / -1: stride-2 layers read a parity-split input (even sizes); 0: NDHWC at the TMA element stride."""
        fusion_set_option(self.handle, FUSION_OPT_CONV_STRIDE2_SPLIT, int(on))

    def conv_slices_per_mma(self, mode):
        """-1: default per layer; 1, 2 or 4: output slices per MMA on every layer."""
        fusion_set_option(self.handle, FUSION_OPT_CONV_SLICES_PER_MMA, int(mode))

    def autotune(self, poses, n_poses=None, on_device=False):
        if n_poses is None:
            n_poses = len(poses["n_lig"])
        fusion_autotune(self.handle, poses, n_poses, on_device)

    def conv_tiles(self):
        return [fusion_describe_conv(self.handle, i) for i in range(self.desc.n_conv)]

    def graph_nodes_per_warp(self, value=None):
        """Set (1, 2, 4, 8; -1 default) and/or return the graph convolution's nodes per warp."""
        if value is not None:
            fusion_set_option(self.handle, FUSION_OPT_GRAPH_NODES_PER_WARP, int(value))
        return fusion_graph_schedule(self.handle)

    def close(self):
        if self.handle:
            fusion_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fusion_server_create(desc: fusion_model_desc, weights, cfg: fusion_server_config) -> C.c_void_p:
    buf = weights if isinstance(weights, (bytes, bytearray)) else np.ascontiguousarray(weights).tobytes()
    h = C.c_void_p()
    cbuf = C.create_string_buffer(bytes(buf), len(buf))
    _check(lib.fusion_server_create(C.byref(desc), cbuf, len(buf), C.byref(cfg), C.byref(h)))
    return h


def fusion_server_submit(server, xyz, feat, n_lig: int) -> int | None:
    """Ticket of the queued pose, or None when the queue is full (FUSION_EAGAIN)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    t = C.c_uint64()
    rc = lib.fusion_server_submit(server, xyz.ctypes.data, feat.ctypes.data, len(xyz), int(n_lig), C.byref(t))
    if rc == FUSION_EAGAIN:
        return None
    _check(rc)
    return t.value


def fusion_server_submit_dtype(server, xyz, feat, n_lig: int, dtype: int) -> int | None:
    """Ticket of the pose queued for a slot of `dtype`, or None when the queue is full (FUSION_EAGAIN)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    t = C.c_uint64()
    rc = lib.fusion_server_submit_dtype(server, xyz.ctypes.data, feat.ctypes.data, len(xyz), int(n_lig), int(dtype),
                                        C.byref(t))
    if rc == FUSION_EAGAIN:
        return None
    _check(rc)
    return t.value


def fusion_server_poll(server, ticket: int):
    """(affinity, latency_s) once scored, else None."""
    a = C.c_float()
    lat = C.c_double()
    rc = lib.fusion_server_poll(server, ticket, C.byref(a), C.byref(lat))
    if rc == FUSION_EAGAIN:
        return None
    _check(rc)
    return a.value, lat.value


def fusion_server_drain(server, timeout_s: float = 600.0) -> None:
    _check(lib.fusion_server_drain(server, timeout_s))


def fusion_server_get_stats(server) -> dict:
    st = fusion_server_stats()
    _check(lib.fusion_server_get_stats(server, C.byref(st)))
    out = {k: getattr(st, k) for k, _ in fusion_server_stats._fields_}
    out["slots_by_dtype"] = {name: int(st.slots_by_dtype[v]) for name, v in DTYPES.items()}
    return out


def fusion_server_destroy(server) -> None:
    lib.fusion_server_destroy(server)


class Server:
    """Continuous-batching server: ``Server(model_dict, weights_blob, max_batch=64, ...)``."""

    def __init__(self, model: dict, weights, max_batch=64, slots=0, batch_window_us=2000.0,
                 hbm_budget_bytes=0, queue_capacity=1 << 20, max_atoms=1200, max_degree=64, dtype=None,
                 dtypes=()):
        """dtypes: further dtypes ("bf16", "fp8", "f32") to run slots of, besides the model's own."""
        self.desc = make_desc(model, max_batch, max_atoms, max_degree, False, dtype)
        mask = 0
        for name in dtypes:
            mask |= 1 << DTYPES[name]
        cfg = fusion_server_config(slots, max_batch, batch_window_us, hbm_budget_bytes, queue_capacity, mask)
        self.handle = fusion_server_create(self.desc, weights, cfg)

    def submit(self, xyz, feat, n_lig, dtype=None):
        if dtype is None:
            return fusion_server_submit(self.handle, xyz, feat, n_lig)
        return fusion_server_submit_dtype(self.handle, xyz, feat, n_lig, DTYPES[dtype])

    def poll(self, ticket):
        return fusion_server_poll(self.handle, ticket)

    def drain(self, timeout_s=600.0):
        fusion_server_drain(self.handle, timeout_s)

    def stats(self):
        return fusion_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            fusion_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
