"""Autotuner for launch geometry.

Sweeps the library's launch knobs (threads per CTA and CTAs per SM of the range
+ CD pass, CTAs per SM of the cooperative saddle rounds, then the stage slack
of the fused decoder or its split form) on a representative field, then the number of parallel branches of the batched CUDA graph on a
mixed batch, timing each setting with CUDA events.  The winners are stored as
JSON and applied with :func:`apply`.  No knob changes an output bit (the tests
compare streams across settings), so tuning is always safe.
"""
from __future__ import annotations

import itertools
import json
import os

import torch

from . import _lib, batch, codec, synth

CACHE = os.environ.get("TOPOSZP_TUNING", os.path.join(os.path.expanduser("~"), ".cache", "toposzp",
                                                       "tuning.json"))
DEFAULT = {"cd_threads": 256, "cd_blocks_per_sm": 8, "rounds_blocks_per_sm": 1, "dec_slack_tiles": 0,
           "batch_branches": 8}


def apply(cfg: dict) -> None:
    t = _lib.Tuning(int(cfg.get("cd_threads", 0)), int(cfg.get("cd_blocks_per_sm", 0)),
                    int(cfg.get("rounds_blocks_per_sm", 0)), int(cfg.get("dec_slack_tiles", 0)),
                    int(cfg.get("saddle_records", 0)), int(cfg.get("dec_split", 0)),
                    int(cfg.get("rank_bitmap", 0)), int(cfg.get("cd_columns", 0)))
    st = _lib.load().toposzp_set_tuning(t)
    if st:
        raise _lib.TopoSZpError(st, "toposzp_set_tuning")


def load() -> dict:
    try:
        with open(CACHE) as f:
            return {**DEFAULT, **json.load(f)}
    except (OSError, ValueError):
        return dict(DEFAULT)


def _time(fn, reps=5) -> float:
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune(side: int = 256, batch_fields: int = 32, save: bool = True, verbose: bool = False) -> dict:
    f = synth.turbulence_3d(side, seed=3, device="cuda")
    out = torch.empty(codec.compress_bound(f.shape), dtype=torch.uint8, device="cuda")
    rec = torch.empty_like(f)

    def step():
        codec.compress_async(f, 1e-3, "rel", out=out)
        codec.decompress_async(out, tuple(f.shape), out=rec)

    best, best_t = dict(DEFAULT), float("inf")
    for th, bps, rb in itertools.product((128, 256, 512), (4, 8, 16), (1, 2, 4)):
        cfg = {"cd_threads": th, "cd_blocks_per_sm": bps, "rounds_blocks_per_sm": rb}
        apply(cfg)
        t = _time(step)
        if verbose:
            print(cfg, round(t, 3))
        if t < best_t:
            best_t, best = t, {**best, **cfg}
    for slack, split in ((16, 0), (64, 0), (256, 0), (1024, 0), (0, 1)):
        cfg = {**best, "dec_slack_tiles": slack, "dec_split": split}
        apply(cfg)
        t = _time(step)
        if verbose:
            print(cfg, round(t, 3))
        if t < best_t:
            best_t, best = t, cfg
    apply(best)
    specs = synth.mixed_batch(count=batch_fields, side2=(128, 2048), side3=(64, 192))
    fields = [s.make("cuda") for s in specs]
    ebs = [s.eb for s in specs]
    bt = {}
    for br in (1, 2, 4, 8, 16):
        plan = batch.BatchPlan.create(fields, ebs, "rel", branches=br).capture()
        bt[br] = _time(lambda: (plan.compress(), plan.decompress()), reps=3)
        del plan
    best["batch_branches"] = min(bt, key=bt.get)
    best["timings_ms"] = {"single_field_best": best_t, "batch_by_branches": bt}
    if save:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as fh:
            json.dump(best, fh, indent=1)
    return best


if __name__ == "__main__":
    import sys
    print(json.dumps(tune(verbose="-v" in sys.argv), indent=1))
