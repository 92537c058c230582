"""Batched form (the native batch plan of the C ABI): many uneven fields
through one CUDA-graph replay give exactly the bytes and values of per-field
plain calls."""
import numpy as np
import pytest
import torch

from paper_2602_17552_gb300 import batch, codec, synth

pytestmark = pytest.mark.gpu


def _fields():
    specs = synth.mixed_batch(count=10, seed=300, side2=(40, 700), side3=(12, 70))
    fs = [s.make("cuda") for s in specs]
    ebs = [s.eb for s in specs]
    return fs, ebs


@pytest.mark.parametrize("branches", [1, 3, 8])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_plain(branches, graph):
    fs, ebs = _fields()
    plan = batch.BatchPlan.create(fs, ebs, "rel", branches=branches)
    if graph:
        plan.capture()
        for _ in range(2):      # replays are repeatable
            plan.compress()
            plan.decompress()
    else:
        plan.run_eager("compress")
        plan.run_eager("decompress")
    plan.check()
    streams = plan.streams_bytes()
    for f, eb, s, it in zip(fs, ebs, streams, plan.items):
        want = codec.compress(f, eb, "rel")
        assert torch.equal(s, want)
        dec = codec.decompress(want, tuple(f.shape))
        assert torch.equal(it.dec.view(torch.int32), dec.view(torch.int32))


@pytest.mark.slow
def test_batch_config4_every_field_equals_plain():
    """The 96-field mixed batch of the batched workload (48 2D fields of side
    128-4096, 48 3D fields of side 64-384, relative bounds 1e-2 to 1e-4,
    about 2.5 GB) through one graph replay: each field's stream bytes and
    decoded values equal those of a plain per-field call."""
    specs = synth.mixed_batch()
    fs = [sp.make("cuda") for sp in specs]
    ebs = [sp.eb for sp in specs]
    plan = batch.BatchPlan.create(fs, ebs, "rel", branches=8).capture()
    plan.compress()
    plan.decompress()
    plan.check()
    for i, (f, eb, got, it) in enumerate(zip(fs, ebs, plan.streams_bytes(), plan.items)):
        want = codec.compress(f, eb, "rel")
        assert torch.equal(got, want), f"field {i} {tuple(f.shape)}: stream differs"
        dec = codec.decompress(want, tuple(f.shape))
        assert torch.equal(it.dec.view(torch.int32), dec.view(torch.int32)), f"field {i}: decoded values differ"


def test_batch_no_topo_and_abs():
    fs, ebs = _fields()
    plan = batch.BatchPlan.create(fs, [1e-2] * len(fs), "abs", branches=4, no_topo=True).capture()
    plan.compress()
    plan.decompress()
    plan.check()
    for f, s, it in zip(fs, plan.streams_bytes(), plan.items):
        want = codec.compress(f, 1e-2, "abs", no_topo=True)
        assert torch.equal(s, want)
        assert torch.equal(it.dec, codec.decompress(want, tuple(f.shape)))


def test_launch_tuning_never_changes_bits():
    from paper_2602_17552_gb300 import autotune
    f3 = synth.turbulence_3d(40, seed=6, device="cuda")
    f2 = synth.climate_2d(300, 640, seed=6, device="cuda")
    want = [codec.compress(f, 1e-3, "rel") for f in (f3, f2)]
    try:
        for th, bps, rb, sl, rec, sp, bm, col, lo in ((128, 4, 1, 1, -1, 0, -1, -1, -1),
                                                      (512, 16, 2, 5000, 1, 1, 0, 0, 0),
                                                      (256, 32, 4, 37, -1, 1, 1, -1, 0),
                                                      (256, 8, 1, 0, 0, 0, 0, 0, -1)):
            autotune.apply({"cd_threads": th, "cd_blocks_per_sm": bps, "rounds_blocks_per_sm": rb,
                            "dec_slack_tiles": sl, "saddle_records": rec, "dec_split": sp, "rank_bitmap": bm,
                            "cd_columns": col, "launch_overlap": lo})
            for f, w in zip((f3, f2), want):
                got = codec.compress(f, 1e-3, "rel")
                assert torch.equal(got, w)
                assert torch.equal(codec.decompress(got, tuple(f.shape)), codec.decompress(w, tuple(f.shape)))
    finally:
        autotune.restore()


def test_batch_inside_a_callers_capture():
    """Under the caller's own stream capture the plan issues its launches
    directly into the caller's graph; replaying that graph gives the same
    streams as plain calls."""
    fs, ebs = _fields()
    plan = batch.BatchPlan.create(fs, ebs, "rel", branches=3).capture()   # warm-up outside capture
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.compress()
            plan.decompress()
    plan.sizes.zero_()
    g.replay()
    plan.check()
    for f, eb, st, it in zip(fs, ebs, plan.streams_bytes(), plan.items):
        want = codec.compress(f, eb, "rel")
        assert torch.equal(st, want)
        assert torch.equal(it.dec, codec.decompress(want, tuple(f.shape)))
