"""Batched compression / decompression of many uneven fields in one launch.

A thin binding of the library's native batch plan (``toposzp_batch_*`` in
``include/toposzp.h``): the plan spreads the fields over parallel branch
streams (longest first onto the least-loaded branch) and replays the whole
batch -- every field's ordinary kernel sequence -- as one CUDA graph.  This
module only allocates the device buffers (torch) and marshals the pointers.

Every field goes through exactly the same kernels as a plain call, so the
compressed bytes and decoded values are identical to per-field runs (checked in
the tests).  ``branches`` comes from the autotuner
(:mod:`paper_2602_17552_gb300.autotune`).  ``run_eager`` issues the same fields
as plain per-field calls, one after another on the current stream: the
baseline the batched form is measured against.
"""
from __future__ import annotations

import ctypes
import json
from dataclasses import dataclass

import torch

from . import _lib, codec


@dataclass
class Item:
    """One field of a batch and its device buffers."""
    shape: tuple
    eb: float
    mode: str
    src: torch.Tensor                 # input field
    out: torch.Tensor = None          # compressed stream buffer (capacity = bound)
    size: torch.Tensor = None         # int64 stream length, written on the device
    st_c: torch.Tensor = None
    st_d: torch.Tensor = None
    dec: torch.Tensor = None          # decoded field


class BatchPlan:
    def __init__(self, items, branches, params, device, handle):
        self.items = items
        self.params = params
        self.device = device
        self._h = handle
        self.branches = int(_lib.load().toposzp_batch_branches(handle))
        n = len(items)
        self.sizes = torch.zeros(n, dtype=torch.int64, device=device)
        self.st_c = torch.zeros(n, dtype=torch.int32, device=device)
        self.st_d = torch.zeros(n, dtype=torch.int32, device=device)
        for i, it in enumerate(items):
            it.size, it.st_c, it.st_d = self.sizes[i:i + 1], self.st_c[i:i + 1], self.st_d[i:i + 1]
        wsb = int(_lib.load().toposzp_batch_workspace_size(handle))
        self.ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=device)
        P = ctypes.c_void_p * n
        self._src = P(*[it.src.data_ptr() for it in items])
        self._out = P(*[it.out.data_ptr() for it in items])
        self._dec = P(*[it.dec.data_ptr() for it in items])
        self._ws_eager = None

    @property
    def nbytes(self) -> int:
        return sum(it.src.numel() * 4 for it in self.items)

    @staticmethod
    def create(fields, ebs, modes="rel", branches: int = 8, no_topo=False, device=None) -> "BatchPlan":
        """fields: list of float32 CUDA tensors (2D or 3D); ebs / modes: per field or scalar."""
        dev = torch.device(device) if device is not None else fields[0].device
        n = len(fields)
        ebs = list(ebs) if isinstance(ebs, (list, tuple)) else [ebs] * n
        modes = list(modes) if isinstance(modes, (list, tuple)) else [modes] * n
        params = codec.make_params(no_topo=no_topo)
        items, ndims, dims, mcodes = [], [], [], []
        for f, eb, md in zip(fields, ebs, modes):
            if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
                raise ValueError("batch fields must be contiguous float32 CUDA tensors")
            nd, d = codec.field_dims(f.shape)
            ndims.append(nd)
            dims.extend(list(_lib.dims3(nd, d)))
            mcodes.append(_lib.EB_REL if md == "rel" else _lib.EB_ABS)
            it = Item(tuple(f.shape), float(eb), md, f)
            it.out = torch.empty(codec.compress_bound(it.shape), dtype=torch.uint8, device=dev)
            it.dec = torch.empty(it.shape, dtype=torch.float32, device=dev)
            items.append(it)
        h = ctypes.c_void_p()
        L = _lib.load()
        st = L.toposzp_batch_plan_create(n, (ctypes.c_int * n)(*ndims), (ctypes.c_uint64 * (3 * n))(*dims),
                                         (ctypes.c_int * n)(*mcodes), (ctypes.c_double * n)(*[it.eb for it in items]),
                                         ctypes.byref(params), json.dumps({"branches": int(branches)}).encode(),
                                         ctypes.byref(h))
        if st:
            raise _lib.TopoSZpError(st, "toposzp_batch_plan_create")
        return BatchPlan(items, branches, params, dev, h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            torch.cuda.synchronize(self.device)
            _lib.load().toposzp_batch_plan_destroy(h)
            self._h = None

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    # ------------------------------------------------------------- running
    def capture(self):
        """Run both directions once: the library captures each direction's CUDA
        graph on its first call with these buffers (later calls replay it)."""
        self.compress()
        self.decompress()
        torch.cuda.synchronize(self.device)
        return self

    def compress(self):
        st = _lib.load().toposzp_batch_compress(self._h, self._src, self._out, self.sizes.data_ptr(),
                                                self.ws.data_ptr(), self.ws.numel(), self.st_c.data_ptr(),
                                                self._stream())
        if st:
            raise _lib.TopoSZpError(st, "toposzp_batch_compress")

    def decompress(self):
        st = _lib.load().toposzp_batch_decompress(self._h, self._out, self._dec, self.ws.data_ptr(),
                                                  self.ws.numel(), self.st_d.data_ptr(), self._stream())
        if st:
            raise _lib.TopoSZpError(st, "toposzp_batch_decompress")

    def run_eager(self, op: str):
        """The same fields as plain per-field calls on the current stream, one
        after another (one workspace shared by all)."""
        if self._ws_eager is None:
            wmax = max(max(codec.compress_workspace_size(it.shape), codec.decompress_workspace_size(it.shape))
                       for it in self.items)
            self._ws_eager = torch.empty(wmax, dtype=torch.uint8, device=self.device)
        for it in self.items:
            if op == "compress":
                codec.compress_async(it.src, it.eb, it.mode, params=self.params, out=it.out, ws=self._ws_eager,
                                     size=it.size, status=it.st_c)
            else:
                codec.decompress_async(it.out, it.shape, out=it.dec, ws=self._ws_eager, status=it.st_d)

    def check(self):
        """Raise if any field's device status is set (synchronises)."""
        torch.cuda.synchronize(self.device)
        for i, (c, d) in enumerate(zip(self.st_c.tolist(), self.st_d.tolist())):
            if c:
                raise _lib.TopoSZpError(c, f"batch item {i} compress")
            if d:
                raise _lib.TopoSZpError(d, f"batch item {i} decompress")

    def streams_bytes(self):
        """Per field: the compressed stream (uint8 CUDA tensor views, exact length)."""
        torch.cuda.synchronize(self.device)
        return [it.out[:int(s)] for it, s in zip(self.items, self.sizes.tolist())]
