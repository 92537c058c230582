"""ctypes binding of libtoposzp.so (the C ABI in include/toposzp.h).

Argument marshalling only.  The shared library is built in-tree by
``paper_2602_17552_gb300.build``; if it is missing this module raises instead of
falling back to any other implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtoposzp.so")

STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "NONFINITE", 3: "EB_TOO_SMALL", 4: "BUFFER_TOO_SMALL",
    5: "CORRUPT_STREAM", 6: "TIMEOUT", 7: "CUDA", 8: "UNSUPPORTED",
}
OK, INVALID_ARG, NONFINITE, EB_TOO_SMALL, BUFFER_TOO_SMALL, CORRUPT_STREAM, TIMEOUT, CUDA, UNSUPPORTED = range(9)
EB_ABS, EB_REL = 0, 1
NO_TOPO = 1
RBF_SOLVE = 2
TILE_BLOCKS = 4


class TopoSZpError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("rs_sweeps", ctypes.c_uint32),
                ("rbf_k", ctypes.c_int32), ("rbf_sigma", ctypes.c_float)]


class Tuning(ctypes.Structure):
    _fields_ = [("cd_threads", ctypes.c_int32), ("cd_blocks_per_sm", ctypes.c_int32),
                ("rounds_blocks_per_sm", ctypes.c_int32), ("dec_slack_tiles", ctypes.c_int32),
                ("saddle_records", ctypes.c_int32), ("dec_split", ctypes.c_int32),
                ("rank_bitmap", ctypes.c_int32), ("cd_columns", ctypes.c_int32),
                ("launch_overlap", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("dims", ctypes.c_uint64 * 3), ("n", ctypes.c_uint64),
                ("total_size", ctypes.c_uint64), ("eps", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("k_min", ctypes.c_uint64), ("k_max", ctypes.c_uint64), ("k_saddle", ctypes.c_uint64),
                ("rbf_k", ctypes.c_int32), ("rbf_sigma", ctypes.c_float)]


EXPORTS = ("toposzp_default_params", "toposzp_status_string", "toposzp_compress_bound",
           "toposzp_compress_workspace_size", "toposzp_decompress_workspace_size", "toposzp_workspace_size",
           "toposzp_compress",
           "toposzp_inspect", "toposzp_decompress", "toposzp_critical_points", "toposzp_topo_errors",
           "toposzp_set_stage_events", "toposzp_set_test_hold", "toposzp_compress_noalloc", "toposzp_noalloc_max_points", "toposzp_set_tuning",
           "toposzp_set_tuning_class", "toposzp_tuning_class", "toposzp_get_tuning",
           "toposzp_batch_plan_create", "toposzp_batch_workspace_size", "toposzp_batch_branches",
           "toposzp_batch_compress", "toposzp_batch_decompress", "toposzp_batch_plan_destroy")

_lib = None


def load() -> ctypes.CDLL:
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'` (there is no fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, c_int, i32p = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
    dims_t = ctypes.POINTER(ctypes.c_uint64)
    L.toposzp_default_params.argtypes = [ctypes.POINTER(Params)]
    L.toposzp_default_params.restype = None
    L.toposzp_status_string.argtypes = [c_int]
    L.toposzp_status_string.restype = ctypes.c_char_p
    for f in ("toposzp_compress_bound", "toposzp_compress_workspace_size", "toposzp_decompress_workspace_size",
              "toposzp_workspace_size"):
        getattr(L, f).argtypes = [c_int, dims_t]
        getattr(L, f).restype = u64
    L.toposzp_compress.argtypes = [vp, c_int, dims_t, c_int, ctypes.c_double, ctypes.POINTER(Params),
                                   vp, u64, vp, vp, u64, i32p, vp]
    L.toposzp_compress.restype = c_int
    L.toposzp_inspect.argtypes = [vp, u64, ctypes.POINTER(Info)]
    L.toposzp_inspect.restype = c_int
    L.toposzp_decompress.argtypes = [vp, u64, vp, u64, vp, u64, i32p, vp]
    L.toposzp_decompress.restype = c_int
    L.toposzp_critical_points.argtypes = [vp, c_int, dims_t, vp, vp, i32p, vp]
    L.toposzp_critical_points.restype = c_int
    L.toposzp_topo_errors.argtypes = [vp, vp, u64, vp, vp]
    L.toposzp_topo_errors.restype = c_int
    L.toposzp_set_stage_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), c_int]
    L.toposzp_set_test_hold.argtypes = [ctypes.c_int32]
    L.toposzp_set_test_hold.restype = c_int
    L.toposzp_set_stage_events.restype = c_int
    L.toposzp_compress_noalloc.argtypes = [vp, c_int, dims_t, c_int, ctypes.c_double, ctypes.POINTER(Params),
                                           vp, u64, vp, i32p, vp]
    L.toposzp_compress_noalloc.restype = c_int
    L.toposzp_set_tuning.argtypes = [ctypes.POINTER(Tuning)]
    L.toposzp_set_tuning.restype = c_int
    L.toposzp_set_tuning_class.argtypes = [c_int, c_int, ctypes.POINTER(Tuning)]
    L.toposzp_set_tuning_class.restype = c_int
    L.toposzp_tuning_class.argtypes = [c_int, dims_t]
    L.toposzp_tuning_class.restype = c_int
    L.toposzp_get_tuning.argtypes = [c_int, dims_t, ctypes.POINTER(Tuning)]
    L.toposzp_get_tuning.restype = c_int
    L.toposzp_noalloc_max_points.argtypes = []
    L.toposzp_noalloc_max_points.restype = u64
    L.toposzp_batch_plan_create.argtypes = [c_int, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(Params), ctypes.c_char_p, ctypes.POINTER(vp)]
    L.toposzp_batch_plan_create.restype = c_int
    L.toposzp_batch_workspace_size.argtypes = [vp]
    L.toposzp_batch_workspace_size.restype = u64
    L.toposzp_batch_branches.argtypes = [vp]
    L.toposzp_batch_branches.restype = c_int
    L.toposzp_batch_compress.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, u64, vp, vp]
    L.toposzp_batch_compress.restype = c_int
    L.toposzp_batch_decompress.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, u64, vp, vp]
    L.toposzp_batch_decompress.restype = c_int
    L.toposzp_batch_plan_destroy.argtypes = [vp]
    L.toposzp_batch_plan_destroy.restype = None
    _lib = L
    apply_tuning_file(L)
    return L


# Launch geometry measured by the autotuner on a GB300 (per dimension and size
# class), committed beside the library and applied when it is loaded.
# TOPOSZP_TUNING names another file; an empty value keeps the defaults.
TUNING_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")
tuning_source = "defaults"


def tuning_struct(cfg: dict) -> Tuning:
    keys = ("cd_threads", "cd_blocks_per_sm", "rounds_blocks_per_sm", "dec_slack_tiles", "saddle_records",
            "dec_split", "rank_bitmap", "cd_columns", "launch_overlap")
    return Tuning(*[int(cfg.get(k, 0)) for k in keys])


def apply_tuning_file(L, path: str = None) -> str:
    """Apply the per-class launch geometry of a tuning file (JSON with a
    "classes" object keyed "2d_0" .. "3d_3"); returns what was applied."""
    global tuning_source
    import json
    path = os.environ.get("TOPOSZP_TUNING", TUNING_FILE) if path is None else path
    if not path or not os.path.exists(path):
        return tuning_source
    with open(path) as f:
        cfg = json.load(f)
    for key, c in cfg.get("classes", {}).items():
        nd, k = int(key[0]), int(key.split("_")[1])
        st = L.toposzp_set_tuning_class(nd, k, ctypes.byref(tuning_struct(c)))
        if st:
            raise TopoSZpError(st, f"toposzp_set_tuning_class {key}")
    tuning_source = os.path.basename(path)
    return tuning_source


def dims3(ndim: int, dims) -> "ctypes.Array":
    d = list(dims) + [1] * (3 - len(dims))
    return (ctypes.c_uint64 * 3)(*[int(x) for x in d[:3]])
