"""Batched compression / decompression of many uneven fields in one launch.

A :class:`BatchPlan` owns device buffers for every field of a batch and
captures the whole batch -- the library's kernel sequence for each field -- as
one CUDA graph.  Fields are spread over ``branches`` parallel graph branches
(longest-first onto the least-loaded branch), so small fields that leave most
SMs idle overlap on the device; each branch reuses one workspace sized for its
largest field.  Replaying the batch is a single ``cudaGraphLaunch``.

Every field goes through exactly the same kernels as a plain call, so the
compressed bytes and decoded values are identical to per-field runs (checked in
the tests).  ``branches`` and the library's launch geometry come from the
autotuner (:mod:`paper_2602_17552_gb300.autotune`).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import torch

from . import _lib, codec


@dataclass
class Item:
    """One field of a batch and its device buffers."""
    shape: tuple
    eb: float
    mode: str
    src: torch.Tensor                 # input field (compress) / decoded output (decompress)
    out: torch.Tensor = None          # compressed stream buffer (capacity = bound)
    size: torch.Tensor = None         # int64 stream length, written on the device
    st_c: torch.Tensor = None
    st_d: torch.Tensor = None
    dec: torch.Tensor = None          # decoded field
    branch: int = 0


@dataclass
class BatchPlan:
    items: list
    branches: int
    params: object
    device: torch.device
    ws_c: list = field(default_factory=list)
    ws_d: list = field(default_factory=list)
    streams: list = field(default_factory=list)
    graph_c: torch.cuda.CUDAGraph = None
    graph_d: torch.cuda.CUDAGraph = None

    @property
    def nbytes(self) -> int:
        return sum(it.src.numel() * 4 for it in self.items)

    # ------------------------------------------------------------ building
    @staticmethod
    def create(fields, ebs, modes="rel", branches: int = 4, no_topo=False, device=None) -> "BatchPlan":
        """fields: list of float32 CUDA tensors (2D or 3D); ebs / modes: per field or scalar."""
        dev = torch.device(device) if device is not None else fields[0].device
        n = len(fields)
        ebs = list(ebs) if isinstance(ebs, (list, tuple)) else [ebs] * n
        modes = list(modes) if isinstance(modes, (list, tuple)) else [modes] * n
        params = codec.make_params(no_topo=no_topo)
        items = []
        for f, eb, md in zip(fields, ebs, modes):
            if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
                raise ValueError("batch fields must be contiguous float32 CUDA tensors")
            items.append(Item(tuple(f.shape), float(eb), md, f))
        branches = max(1, min(int(branches), n))
        # longest first onto the least-loaded branch
        load = [0] * branches
        for it in sorted(items, key=lambda it: -it.src.numel()):
            b = min(range(branches), key=lambda j: load[j])
            it.branch = b
            load[b] += it.src.numel()
        plan = BatchPlan(items, branches, params, dev)
        for b in range(branches):
            mine = [it for it in items if it.branch == b]
            wc = max((codec.compress_workspace_size(it.shape) for it in mine), default=256)
            wd = max((codec.decompress_workspace_size(it.shape) for it in mine), default=256)
            plan.ws_c.append(torch.empty(wc, dtype=torch.uint8, device=dev))
            plan.ws_d.append(torch.empty(wd, dtype=torch.uint8, device=dev))
            plan.streams.append(torch.cuda.Stream(device=dev))
        for it in items:
            it.out = torch.empty(codec.compress_bound(it.shape), dtype=torch.uint8, device=dev)
            it.size = torch.zeros(1, dtype=torch.int64, device=dev)
            it.st_c = torch.zeros(1, dtype=torch.int32, device=dev)
            it.st_d = torch.zeros(1, dtype=torch.int32, device=dev)
            it.dec = torch.empty(it.shape, dtype=torch.float32, device=dev)
        return plan

    def _enqueue(self, op: str):
        """Issue the batch on the branch streams, forked from and joined into the
        current stream (works eagerly and under graph capture)."""
        main = torch.cuda.current_stream(self.device)
        fork = torch.cuda.Event()
        fork.record(main)
        joins = []
        for b, s in enumerate(self.streams):
            s.wait_event(fork)
            with torch.cuda.stream(s):
                for it in self.items:
                    if it.branch != b:
                        continue
                    if op == "compress":
                        codec.compress_async(it.src, it.eb, it.mode, params=self.params, out=it.out,
                                             ws=self.ws_c[b], size=it.size, status=it.st_c, stream=s)
                    else:
                        codec.decompress_async(it.out, it.shape, out=it.dec, ws=self.ws_d[b],
                                               status=it.st_d, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
            joins.append(ev)
        for ev in joins:
            main.wait_event(ev)

    def capture(self):
        """Capture compress and decompress of the whole batch as two CUDA graphs."""
        self.run_eager("compress")       # warm-up outside capture (lazy init, occupancy queries)
        self.run_eager("decompress")
        torch.cuda.synchronize(self.device)
        self.graph_c = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph_c):
            self._enqueue("compress")
        self.graph_d = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph_d):
            self._enqueue("decompress")
        return self

    # ------------------------------------------------------------- running
    def run_eager(self, op: str):
        self._enqueue(op)

    def compress(self):
        """Replay the compress graph (one launch) on the current stream."""
        if self.graph_c is None:
            self.run_eager("compress")
        else:
            self.graph_c.replay()

    def decompress(self):
        if self.graph_d is None:
            self.run_eager("decompress")
        else:
            self.graph_d.replay()

    def check(self):
        """Raise if any field's device status is set (synchronises)."""
        torch.cuda.synchronize(self.device)
        for i, it in enumerate(self.items):
            for st, what in ((it.st_c, "compress"), (it.st_d, "decompress")):
                v = int(st.item())
                if v:
                    raise _lib.TopoSZpError(v, f"batch item {i} {what}")

    def streams_bytes(self):
        """Per field: the compressed stream (uint8 CUDA tensor views, exact length)."""
        torch.cuda.synchronize(self.device)
        return [it.out[:int(it.size.item())] for it in self.items]
