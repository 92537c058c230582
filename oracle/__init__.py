"""TopoSZp CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python wrapper (ctypes + numpy) around the plain single-threaded C oracle in
``toposzp_oracle.c``.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the library itself never
does.  The C source is compiled on first use (or by ``build()``) with
``-O2 -ffp-contract=off -fno-fast-math`` so that every floating-point operation
is a single IEEE-754 operation rounded to nearest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "toposzp_oracle.c")
_HDR = os.path.join(_HERE, "toposzp_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, INVALID_ARG, NONFINITE, EB_TOO_SMALL, BUFFER_TOO_SMALL, CORRUPT = range(6)
R, MIN, SAD, MAX = 0, 1, 2, 3
NO_TOPO = 1
RBF_SOLVE = 2
TILE_BLOCKS = 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` next to its source."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.orc_compress.restype = ctypes.c_int
        L.orc_compress.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32, ctypes.c_float,
                                   ctypes.c_void_p, ctypes.c_uint64, u64p]
        L.orc_decompress.restype = ctypes.c_int
        L.orc_decompress.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_compress_bound.restype = ctypes.c_uint64
        L.orc_compress_bound.argtypes = [ctypes.c_int, u64p]
        L.orc_tile_blocks.restype = ctypes.c_uint64
        L.orc_tile_blocks.argtypes = [ctypes.c_int, u64p]
        L.orc_critical_points.restype = None
        L.orc_critical_points.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_void_p]
        L.orc_classify.restype = ctypes.c_int
        L.orc_classify.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_uint64]
        L.orc_qparams_compute.restype = ctypes.c_int
        L.orc_qparams_compute.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_void_p]
        L.orc_quantize.restype = ctypes.c_int32
        L.orc_quantize.argtypes = [ctypes.c_float, ctypes.c_void_p]
        L.orc_dequantize.restype = ctypes.c_float
        L.orc_dequantize.argtypes = [ctypes.c_int32, ctypes.c_void_p]
        L.orc_ranks.restype = ctypes.c_uint64
        L.orc_ranks.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                ctypes.c_void_p]
        L.orc_exp_neg.restype = ctypes.c_double
        L.orc_exp_neg.argtypes = [ctypes.c_double]
        L.orc_rbf_solve.restype = ctypes.c_int
        L.orc_rbf_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_void_p]
        L.orc_colour.restype = ctypes.c_int
        L.orc_colour.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.POINTER(ctypes.c_int)]
        L.orc_topo_errors.restype = None
        L.orc_topo_errors.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        _lib = L
    return _lib


class QParams(ctypes.Structure):
    _fields_ = [("vmin", ctypes.c_float), ("vmax", ctypes.c_float), ("eps", ctypes.c_double),
                ("w_f", ctypes.c_float), ("r_f", ctypes.c_float), ("h_f", ctypes.c_float),
                ("const_field", ctypes.c_int)]


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def _dims3(a: np.ndarray):
    """(ndim, dims[3]) with dims[0] the fastest axis, from a C-ordered array."""
    if a.ndim == 2:
        return 2, (ctypes.c_uint64 * 3)(a.shape[1], a.shape[0], 1)
    if a.ndim == 3:
        return 3, (ctypes.c_uint64 * 3)(a.shape[2], a.shape[1], a.shape[0])
    raise ValueError("field must be 2D or 3D")


def _f32(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a


def qparams(a, rel: bool, eb: float) -> QParams:
    a = _f32(a)
    p = QParams()
    st = lib().orc_qparams_compute(a.ctypes.data, a.size, int(rel), float(eb), ctypes.byref(p))
    if st:
        raise OracleError(st, "qparams")
    return p


def quantize(a, p: QParams) -> np.ndarray:
    a = _f32(a).ravel()
    f = lib().orc_quantize
    return np.array([f(float(v), ctypes.byref(p)) for v in a], dtype=np.int32)


def dequantize(q, p: QParams) -> np.ndarray:
    f = lib().orc_dequantize
    return np.array([f(int(v), ctypes.byref(p)) for v in np.asarray(q).ravel()], dtype=np.float32)


def critical_points(a) -> np.ndarray:
    """Per-point labels r=0, m=1, s=2, M=3 (uint8, same shape as ``a``)."""
    a = _f32(a)
    nd, d3 = _dims3(a)
    out = np.empty(a.shape, np.uint8)
    lib().orc_critical_points(a.ctypes.data, nd, d3, out.ctypes.data)
    return out


def classify(a, i: int) -> int:
    a = _f32(a)
    nd, d3 = _dims3(a)
    return lib().orc_classify(a.ctypes.data, nd, d3, int(i))


def ranks(a, labels, p: QParams) -> np.ndarray:
    a = _f32(a)
    lab = np.ascontiguousarray(labels, dtype=np.uint8)
    out = np.zeros(a.size + 1, np.int32)
    k = lib().orc_ranks(a.ctypes.data, lab.ctypes.data, a.size, ctypes.byref(p), out.ctypes.data)
    return out[:k].copy()


def exp_neg(t: float) -> float:
    return lib().orc_exp_neg(float(t))


def rbf_solve(ndim: int, r: int, sigma: float, at=(0, 0, 0)) -> np.ndarray:
    """Weights of the RBF interpolant with a constant term over N_r(p) minus
    p, evaluated at offset `at` (x, y, z) from p, in the offset table order
    ((z, y, x) ascending; binary64)."""
    out = np.zeros(343, np.float64)
    m = lib().orc_rbf_solve(ndim, r, float(sigma), int(at[0]), int(at[1]), int(at[2]), out.ctypes.data)
    return out[:m].copy()


def colour(ndim: int, x: int, y: int, z: int = 0):
    nc = ctypes.c_int(0)
    c = lib().orc_colour(ndim, x, y, z, ctypes.byref(nc))
    return c, nc.value


def compress_bound(shape) -> int:
    a = np.empty(shape, np.uint8)
    nd, d3 = _dims3(a)
    return int(lib().orc_compress_bound(nd, d3))


def tile_blocks(shape) -> int:
    """Number of format-v2 (tile-shaped) blocks covering a grid of `shape`."""
    a = np.empty(shape, np.uint8)
    nd, d3 = _dims3(a)
    return int(lib().orc_tile_blocks(nd, d3))


def compress(a, eb: float, rel: bool = True, no_topo: bool = False, rs_sweeps: int = 1,
             rbf_k: int = 0, rbf_sigma: float = 0.0, rbf_solve: bool = False, tile_blocks: bool = False) -> bytes:
    a = _f32(a)
    nd, d3 = _dims3(a)
    cap = int(lib().orc_compress_bound(nd, d3))
    out = np.empty(cap, np.uint8)
    size = ctypes.c_uint64(0)
    flags = ((NO_TOPO if no_topo else 0) | (RBF_SOLVE if rbf_solve else 0) |
             (TILE_BLOCKS if tile_blocks else 0))
    st = lib().orc_compress(a.ctypes.data, nd, d3, int(rel), float(eb), flags,
                            int(rs_sweeps), int(rbf_k), float(rbf_sigma), out.ctypes.data, cap,
                            ctypes.byref(size))
    if st:
        raise OracleError(st, "compress")
    return out[:size.value].tobytes()


def decompress(buf: bytes, shape, stages: bool = False):
    """Decoded field; with ``stages`` also (D0 after QZ^, D1 after the extrema
    stencils, stats = [extrema restored, extrema skipped by the bound, saddles fixed, 0])."""
    src = np.frombuffer(buf, np.uint8)
    n = int(np.prod(shape))
    out = np.empty(shape, np.float32)
    d0 = np.empty(shape, np.float32) if stages else None
    d1 = np.empty(shape, np.float32) if stages else None
    stats = np.zeros(4, np.uint64)
    st = lib().orc_decompress(src.ctypes.data, src.size, out.ctypes.data, n,
                              d0.ctypes.data if stages else None, d1.ctypes.data if stages else None,
                              stats.ctypes.data)
    if st:
        raise OracleError(st, "decompress")
    if stages:
        return out, d0, d1, stats
    return out


def topo_errors(lab_a, lab_b) -> np.ndarray:
    """Counts [kind, type] with kind 0 FN, 1 FP, 2 FT and type r/m/s/M."""
    a = np.ascontiguousarray(lab_a, np.uint8).ravel()
    b = np.ascontiguousarray(lab_b, np.uint8).ravel()
    out = np.zeros(12, np.uint64)
    lib().orc_topo_errors(a.ctypes.data, b.ctypes.data, a.size, out.ctypes.data)
    return out.reshape(3, 4)


# ------------------------------------------------------------ stream parsing

HEADER_FIELDS = {
    "magic": (0, "<u4"), "version": (4, "<u4"), "ndim": (8, "<u4"), "L": (12, "<u4"),
    "nx": (16, "<u8"), "ny": (24, "<u8"), "nz": (32, "<u8"), "flags": (40, "<u4"),
    "rel": (44, "<u4"), "eb": (48, "<f8"), "eps": (56, "<f8"), "w_f": (64, "<f4"),
    "r_f": (68, "<f4"), "h_f": (72, "<f4"), "const_field": (76, "<u4"), "vmin": (80, "<f4"),
    "vmax": (84, "<f4"), "rbf_k": (88, "<u4"), "rbf_sigma": (92, "<f4"), "rs_sweeps": (96, "<u4"),
    "n": (104, "<u8"), "nb": (112, "<u8"), "k_min": (120, "<u8"), "k_max": (128, "<u8"),
    "k_sad": (136, "<u8"), "sum_abs": (144, "<u8"), "off_s1": (152, "<u8"), "off_s2": (160, "<u8"),
    "off_s4": (168, "<u8"), "off_s6": (176, "<u8"), "off_s5": (184, "<u8"), "off_s7": (192, "<u8"),
    "total": (200, "<u8"), "pay_words": (208, "<u8"), "rank_pay_words": (216, "<u4"),
}


def header(buf: bytes) -> dict:
    b = np.frombuffer(buf[:256], np.uint8)
    out = {}
    for k, (off, dt) in HEADER_FIELDS.items():
        size = np.dtype(dt).itemsize
        out[k] = np.frombuffer(b[off:off + size].tobytes(), dt)[0].item()
    out["g"] = np.frombuffer(b[220:256].tobytes(), "<f4").copy()
    return out
