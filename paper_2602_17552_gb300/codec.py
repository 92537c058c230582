"""Torch-facing wrappers of the TopoSZp C ABI.

Tensors supply device memory; ``torch.cuda.current_stream()`` (or an explicit
stream) orders the work.  Every step of compression and decompression runs in
the library's CUDA kernels; this module only sizes buffers, passes pointers and
reads back status words.

Shapes: a 2D field is ``(ny, nx)``, a 3D field ``(nz, ny, nx)``; ``dims`` passed
to the library are ``(nx, ny[, nz])`` with x fastest.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import EB_ABS, EB_REL, NO_TOPO, RBF_SOLVE, TILE_BLOCKS, TopoSZpError

_WS = {}   # (device, kind) -> cached workspace tensor (grown on demand)


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def field_dims(shape):
    """(ndim, dims) with dims[0] = nx the fastest axis."""
    if len(shape) == 2:
        return 2, (shape[1], shape[0])
    if len(shape) == 3:
        return 3, (shape[2], shape[1], shape[0])
    raise ValueError("fields are 2D (ny, nx) or 3D (nz, ny, nx)")


def compress_bound(shape) -> int:
    nd, d = field_dims(shape)
    return int(_lib.load().toposzp_compress_bound(nd, _lib.dims3(nd, d)))


def compress_workspace_size(shape) -> int:
    nd, d = field_dims(shape)
    return int(_lib.load().toposzp_compress_workspace_size(nd, _lib.dims3(nd, d)))


def decompress_workspace_size(shape) -> int:
    nd, d = field_dims(shape)
    return int(_lib.load().toposzp_decompress_workspace_size(nd, _lib.dims3(nd, d)))


def workspace(kind: str, nbytes: int, device) -> torch.Tensor:
    """A cached uint8 device buffer of at least ``nbytes`` (one per device and kind).
    Callers that overlap calls on several streams must pass their own buffers."""
    key = (torch.device(device).index, kind)
    buf = _WS.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _WS[key] = buf
    return buf


def make_params(no_topo=False, rs_sweeps=1, rbf_k=0, rbf_sigma=0.0, rbf_solve=False,
                tile_blocks=False) -> _lib.Params:
    p = _lib.Params()
    _lib.load().toposzp_default_params(ctypes.byref(p))
    p.flags = ((NO_TOPO if no_topo else 0) | (RBF_SOLVE if rbf_solve else 0) |
               (TILE_BLOCKS if tile_blocks else 0))
    p.rs_sweeps = int(rs_sweeps)
    p.rbf_k = int(rbf_k)
    p.rbf_sigma = float(rbf_sigma)
    return p


def _check(st: int, where: str):
    if st != 0:
        raise TopoSZpError(st, where)


def _check_field(field: torch.Tensor):
    if not (field.is_cuda and field.dtype == torch.float32 and field.is_contiguous()):
        raise ValueError("field must be a contiguous float32 CUDA tensor")


@dataclass
class CompressCall:
    """Buffers of one asynchronous compression: ``out`` holds the stream, its
    length lands in ``size`` and the device status in ``status`` (both int64 /
    int32 device tensors, valid once the stream has reached them)."""
    out: torch.Tensor
    size: torch.Tensor
    status: torch.Tensor


def compress_async(field: torch.Tensor, eb: float, mode: str = "rel", *, params=None, out=None,
                   ws=None, size=None, status=None, stream=None) -> CompressCall:
    """Queue one compression on ``stream``; no host synchronisation."""
    _check_field(field)
    nd, d = field_dims(field.shape)
    L = _lib.load()
    dims = _lib.dims3(nd, d)
    dev = field.device
    if out is None:
        out = torch.empty(int(L.toposzp_compress_bound(nd, dims)), dtype=torch.uint8, device=dev)
    if ws is None:
        ws = workspace("compress", int(L.toposzp_compress_workspace_size(nd, dims)), dev)
    if size is None:
        size = torch.zeros(1, dtype=torch.int64, device=dev)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=dev)
    p = params if params is not None else make_params()
    st = L.toposzp_compress(field.data_ptr(), nd, dims, EB_REL if mode == "rel" else EB_ABS, float(eb),
                            ctypes.byref(p), out.data_ptr(), out.numel(), size.data_ptr(), ws.data_ptr(),
                            ws.numel(), status.data_ptr(), _stream_handle(stream))
    _check(st, "toposzp_compress")
    return CompressCall(out, size, status)


def compress(field: torch.Tensor, eb: float, mode: str = "rel", *, no_topo=False, rs_sweeps=1, rbf_k=0,
             rbf_sigma=0.0, rbf_solve=False, tile_blocks=False, stream=None) -> torch.Tensor:
    """Compress and return the stream as a uint8 CUDA tensor of its exact length
    (synchronises ``stream`` to read the length and the device status).
    ``rbf_solve`` selects the literal RBF interpolation for the decoder's
    saddle refinement (stored in the stream's header); ``tile_blocks`` writes
    format v2 (tile-shaped blocks; the same decoded field, a smaller stream
    on most fields)."""
    call = compress_async(field, eb, mode,
                          params=make_params(no_topo, rs_sweeps, rbf_k, rbf_sigma, rbf_solve, tile_blocks),
                          stream=stream)
    (torch.cuda.current_stream() if stream is None else stream).synchronize()
    _check(int(call.status.item()), "toposzp_compress (device)")
    return call.out[:int(call.size.item())]


def inspect(stream_bytes) -> _lib.Info:
    """Parse a stream header; accepts a CUDA or CPU uint8 tensor, or bytes."""
    if isinstance(stream_bytes, torch.Tensor):
        hdr = stream_bytes[:256].cpu().numpy().tobytes()
    else:
        hdr = bytes(stream_bytes[:256])
    info = _lib.Info()
    buf = ctypes.create_string_buffer(hdr, len(hdr))
    _check(_lib.load().toposzp_inspect(buf, len(hdr), ctypes.byref(info)), "toposzp_inspect")
    return info


def shape_of(info: _lib.Info):
    d = list(info.dims)
    return (d[1], d[0]) if info.ndim == 2 else (d[2], d[1], d[0])


def decompress_async(stream_bytes: torch.Tensor, shape, *, out=None, ws=None, status=None,
                     stream=None):
    """Queue one decompression; returns (out, status).  ``shape`` must be the
    field's shape (the kernels check it against the header on the device)."""
    nd, d = field_dims(shape)
    L = _lib.load()
    n = 1
    for s in shape:
        n *= int(s)
    dev = stream_bytes.device
    if out is None:
        out = torch.empty(tuple(shape), dtype=torch.float32, device=dev)
    if ws is None:
        ws = workspace("decompress", int(L.toposzp_decompress_workspace_size(nd, _lib.dims3(nd, d))), dev)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=dev)
    st = L.toposzp_decompress(stream_bytes.data_ptr(), stream_bytes.numel(), out.data_ptr(), n,
                              ws.data_ptr(), ws.numel(), status.data_ptr(), _stream_handle(stream))
    _check(st, "toposzp_decompress")
    return out, status


def decompress(stream_bytes: torch.Tensor, shape=None, *, stream=None) -> torch.Tensor:
    """Decompress a stream (uint8 CUDA tensor).  Without ``shape`` the header is
    read back to the host first."""
    if shape is None:
        shape = shape_of(inspect(stream_bytes))
    out, status = decompress_async(stream_bytes, shape, stream=stream)
    (torch.cuda.current_stream() if stream is None else stream).synchronize()
    _check(int(status.item()), "toposzp_decompress (device)")
    return out


def critical_points(field: torch.Tensor, *, stream=None, counts=True):
    """Section IV-A(1) labels of any field: (packed uint32 labels as an int32
    tensor of ceil(n/16) words, counts of r/m/s/M as an int64 tensor)."""
    if not (field.is_cuda and field.dtype == torch.float32 and field.is_contiguous()):
        raise ValueError("field must be a contiguous float32 CUDA tensor")
    nd, d = field_dims(field.shape)
    n = field.numel()
    labels = torch.empty((n + 15) // 16, dtype=torch.int32, device=field.device)
    cnt = torch.zeros(4, dtype=torch.int64, device=field.device) if counts else None
    status = torch.zeros(1, dtype=torch.int32, device=field.device)
    st = _lib.load().toposzp_critical_points(field.data_ptr(), nd, _lib.dims3(nd, d), labels.data_ptr(),
                                             cnt.data_ptr() if counts else None, status.data_ptr(),
                                             _stream_handle(stream))
    _check(st, "toposzp_critical_points")
    return labels, cnt


def topo_errors(labels_a: torch.Tensor, labels_b: torch.Tensor, n: int, *, stream=None) -> torch.Tensor:
    """FN / FP / FT counts (3 x 4, int64) between two packed label maps."""
    out = torch.zeros(12, dtype=torch.int64, device=labels_a.device)
    st = _lib.load().toposzp_topo_errors(labels_a.data_ptr(), labels_b.data_ptr(), int(n), out.data_ptr(),
                                         _stream_handle(stream))
    _check(st, "toposzp_topo_errors")
    return out.view(3, 4)


def tradeoff(field: torch.Tensor, eb: float, mode: str = "rel", *, no_topo=False, rbf_solve=False,
             tile_blocks=False, labels=None, stream=None) -> dict:
    """One point of the bit-rate / topology-error trade-off (Section III-B,
    Table II): compress and decompress ``field`` and count the false
    negatives, false positives and false types of the decompressed field's
    critical points against the original's (Section IV-A(1) labels), per type
    in the order r, m, s, M (FN and FT by the original type, FP by the new).
    ``labels``: the original's packed labels, if already computed.
    Returns bytes, bit_rate (bits per value), ratio, max_err_over_eps (the
    largest |decoded - input| over the stream's absolute bound), fn, fp, ft."""
    n = field.numel()
    if labels is None:
        labels, _ = critical_points(field, counts=False, stream=stream)
    buf = compress(field, eb, mode, no_topo=no_topo, rbf_solve=rbf_solve, tile_blocks=tile_blocks, stream=stream)
    info = inspect(buf)
    dec = decompress(buf, tuple(field.shape), stream=stream)
    lab_d, _ = critical_points(dec, counts=False, stream=stream)
    e = topo_errors(labels, lab_d, n, stream=stream).cpu().tolist()
    err = float((dec.double() - field.double()).abs().max())
    return {"bytes": int(buf.numel()), "bit_rate": 8.0 * buf.numel() / n, "ratio": 4.0 * n / buf.numel(),
            "max_err_over_eps": err / info.eps, "fn": e[0], "fp": e[1], "ft": e[2]}


def unpack_labels(words: torch.Tensor, n: int) -> torch.Tensor:
    """Packed 2-bit labels -> one uint8 per point (any device)."""
    w = words.to(torch.int64) & 0xFFFFFFFF
    shifts = torch.arange(0, 32, 2, device=w.device)
    lab = (w.unsqueeze(1) >> shifts) & 3
    return lab.reshape(-1)[:n].to(torch.uint8)
