"""Serving: a continuous-batching request loop over the TopoSZp C ABI.

Requests (compress a field / decompress a stream) arrive on a Poisson clock,
as in-situ simulation output would, with their inputs already resident in HBM
(produced before the clock starts; for decompress requests the stream is made
beforehand, untimed).  The loop

* reserves one device arena (a fraction of the free HBM seen at start) and
  carves each request's workspace and output out of it with a first-fit free
  list -- admission by free HBM: an arrived request is admitted, in arrival
  order, as soon as a stream slot is free and its buffers fit in the arena;
* runs every admitted request on a stream of its own, so requests that arrive
  while others are on the GPU overlap with them on the device;
* polls completion events; latency = completion - arrival (host clock), and
  frees the request's arena space.

``serial=True`` serves the same stream one request at a time (the plain
per-request baseline).  Neither mode changes a single output bit.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import codec, synth

ALIGN = 256


class Arena:
    """First-fit allocator over one preallocated device buffer (host-side
    bookkeeping only; device memory is never freed or reallocated)."""

    def __init__(self, nbytes: int, device):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.size = nbytes
        self.free = [(0, nbytes)]   # sorted (offset, length)

    def alloc(self, n: int):
        n = (n + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                return off, n
        return None

    def release(self, off: int, n: int):
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    def view(self, off: int, n: int) -> torch.Tensor:
        return self.buf[off:off + n]

    @property
    def free_bytes(self) -> int:
        return sum(ln for _, ln in self.free)


@dataclass
class Job:
    req: synth.Request
    shape: tuple
    inp: torch.Tensor = None          # field (compress) or stream (decompress)
    ws_bytes: int = 0
    out_bytes: int = 0
    lease: tuple = None
    t_start: float = None
    t_done: float = None
    out: torch.Tensor = None
    size: torch.Tensor = None
    status: torch.Tensor = None
    done_ev: torch.cuda.Event = None
    stream: torch.cuda.Stream = None


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    bytes_total: int = 0
    wall_s: float = 0.0
    max_inflight: int = 0
    admitted_waits: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": len(self.latencies_ms), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "aggregate_gbs": self.bytes_total / max(self.wall_s, 1e-9) / 1e9,
                "wall_s": self.wall_s, "max_inflight": self.max_inflight,
                "memory_waits": self.admitted_waits}


def _sizes(shape, op: str):
    n = int(np.prod(shape))
    if op == "compress":
        return codec.compress_workspace_size(shape), codec.compress_bound(shape)
    return codec.decompress_workspace_size(shape), 4 * n


def _bytes_needed(shape, op: str) -> int:
    ws, out = _sizes(shape, op)
    return (ws + ALIGN - 1) // ALIGN * ALIGN + (out + ALIGN - 1) // ALIGN * ALIGN


class Server:
    def __init__(self, device="cuda", slots: int = 8, hbm_fraction: float = 0.5, arena_bytes: int = None,
                 keep_outputs: bool = False):
        self.device = torch.device(device)
        self.slots = slots
        if arena_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            arena_bytes = int(free * hbm_fraction)
        self.arena = Arena(arena_bytes, self.device)
        self.keep_outputs = keep_outputs
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]

    @property
    def budget(self) -> int:
        return self.arena.size

    @budget.setter
    def budget(self, nbytes: int):
        self.arena = Arena(nbytes, self.device)

    # ---------------------------------------------------------- production
    def produce(self, jobs):
        """Inputs for every request, resident before the clock starts."""
        for j in jobs:
            spec = j.req.spec
            f = spec.make(self.device)
            if j.req.op == "compress":
                j.inp = f
            else:
                j.inp = codec.compress(f, spec.eb, "rel").clone()
        torch.cuda.synchronize(self.device)

    # -------------------------------------------------------------- serving
    def _launch(self, j: Job, stream: torch.cuda.Stream):
        spec = j.req.spec
        j.stream = stream
        # the job's input, size and status words were written on the current
        # stream: order the slot stream after them, and tell the caching
        # allocator that the slot stream uses them
        stream.wait_stream(torch.cuda.current_stream(self.device))
        for t in (j.inp, j.size, j.status):
            t.record_stream(stream)
        off, ln = j.lease
        ws = self.arena.view(off, j.ws_bytes)
        wsa = (j.ws_bytes + ALIGN - 1) // ALIGN * ALIGN
        out = self.arena.view(off + wsa, j.out_bytes)
        if j.req.op == "compress":
            call = codec.compress_async(j.inp, spec.eb, "rel", out=out, ws=ws, stream=stream,
                                        size=j.size, status=j.status)
            j.out = call.out
        else:
            j.out, _ = codec.decompress_async(j.inp, j.shape, out=out.view(torch.float32).view(j.shape), ws=ws,
                                              status=j.status, stream=stream)
        j.done_ev.record(stream)

    def run(self, requests, serial: bool = False, produced: list = None, keep=None) -> tuple:
        """Serve `requests` (synth.Request list sorted by arrival).  Returns
        (ServeStats, outputs); outputs[rid] is the compressed stream or decoded
        field (CPU copy) when keep_outputs is set, or for the request ids in
        `keep` when given."""
        jobs = produced if produced is not None else [Job(r, r.spec.shape()) for r in requests]
        for j in jobs:
            j.ws_bytes, j.out_bytes = _sizes(j.shape, j.req.op)
            if _bytes_needed(j.shape, j.req.op) > self.arena.size:
                raise MemoryError(f"request {j.req.rid} does not fit the arena")
            j.size = torch.zeros(1, dtype=torch.int64, device=self.device)
            j.status = torch.zeros(1, dtype=torch.int32, device=self.device)
            j.done_ev = torch.cuda.Event()
        if produced is None:
            self.produce(jobs)
        stats = ServeStats()
        outputs = {}
        waiting = list(jobs)
        inflight = []
        free_streams = list(self.streams)
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        first_arrival = jobs[0].req.t_arrive if jobs else 0.0
        while waiting or inflight:
            # admit arrived requests in order while a slot and arena space are free
            while waiting and waiting[0].req.t_arrive <= clock() and free_streams:
                if serial and inflight:
                    break
                j = waiting[0]
                lease = self.arena.alloc(_bytes_needed(j.shape, j.req.op))
                if lease is None:
                    stats.admitted_waits += 1
                    break
                waiting.pop(0)
                j.lease = lease
                j.t_start = clock()
                self._launch(j, free_streams.pop())
                inflight.append(j)
                stats.max_inflight = max(stats.max_inflight, len(inflight))
            still = []
            for j in inflight:
                if j.done_ev.query():
                    j.t_done = clock()
                    st = int(j.status.item())
                    if st:
                        raise RuntimeError(f"request {j.req.rid} failed with status {st}")
                    stats.latencies_ms.append(1e3 * (j.t_done - j.req.t_arrive))
                    stats.bytes_total += 4 * int(np.prod(j.shape))
                    if (keep is None and self.keep_outputs) or (keep is not None and j.req.rid in keep):
                        if j.req.op == "compress":
                            outputs[j.req.rid] = j.out[:int(j.size.item())].cpu()
                        else:
                            outputs[j.req.rid] = j.out.cpu()
                    self.arena.release(*j.lease)
                    free_streams.append(j.stream)
                    j.out = None
                else:
                    still.append(j)
            inflight = still
            if not inflight and waiting:
                dt = waiting[0].req.t_arrive - clock()
                if dt > 0:
                    time.sleep(min(dt, 1e-3))
            elif inflight:
                time.sleep(1e-5)
        torch.cuda.synchronize(self.device)
        stats.wall_s = clock() - first_arrival
        return stats, outputs


def retimed(jobs, rate_hz: float, gaps):
    """The same requests (and resident inputs) with arrival times from the
    unit-rate inter-arrival gaps scaled to `rate_hz` (inf: all at once)."""
    out, t = [], 0.0
    for j, g in zip(jobs, gaps):
        t = 0.0 if rate_hz == float("inf") else t + g / rate_hz
        r = synth.Request(j.req.rid, t, j.req.op, j.req.spec)
        out.append(Job(r, j.shape, inp=j.inp))
    return out


def plain_result(req: synth.Request, device="cuda"):
    """The same request served alone through the plain entry points."""
    f = req.spec.make(device)
    if req.op == "compress":
        return codec.compress(f, req.spec.eb, "rel").cpu()
    buf = codec.compress(f, req.spec.eb, "rel")
    return codec.decompress(buf, req.spec.shape()).cpu()
