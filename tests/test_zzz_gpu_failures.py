"""Failure paths on the GPU without a fault, trap or hang: a bounded device wait
that runs out ends the call with TOPOSZP_ERR_TIMEOUT in its status word, and
the next call on the same context decodes normally."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2602_17552_gb300 import _lib, codec, synth

pytestmark = pytest.mark.gpu


def test_wait_that_runs_out_reports_timeout():
    a = synth.turbulence_3d(32, seed=1).numpy()   # 32768 points: four decode tiles
    f = torch.from_numpy(a).cuda()
    buf = codec.compress(f, 1e-3, "rel")
    lib = _lib.load()
    # tile 0 never publishes its decode stage: every wait for it gives up
    assert lib.toposzp_set_test_hold(0) == _lib.OK
    try:
        with pytest.raises(_lib.TopoSZpError) as ei:
            codec.decompress(buf, a.shape)
        assert ei.value.status == _lib.TIMEOUT
    finally:
        assert lib.toposzp_set_test_hold(-1) == _lib.OK
    out = codec.decompress(buf, a.shape).cpu().numpy()
    want = oracle.decompress(buf.cpu().numpy().tobytes(), a.shape)
    assert np.array_equal(out.view(np.uint32), want.view(np.uint32))


def test_one_wait_running_out_ends_the_call_quickly():
    """With many more virtual tiles than resident CTAs (a 128^3 field: 256
    decode tiles plus the trailing stage slots), a held tile must not make
    every dependent wait run its full limit in turn: once the first wait
    gives up and sets the status word, the others stop waiting.  One wait's
    limit is about a second; the whole call must end within a few."""
    a = synth.turbulence_3d(128, seed=2).numpy()
    f = torch.from_numpy(a).cuda()
    buf = codec.compress(f, 1e-3, "rel")
    codec.decompress(buf, a.shape)            # warm: the timing below is the waits only
    torch.cuda.synchronize()
    lib = _lib.load()
    assert lib.toposzp_set_test_hold(3) == _lib.OK
    try:
        t0 = time.perf_counter()
        with pytest.raises(_lib.TopoSZpError) as ei:
            codec.decompress(buf, a.shape)
        dt = time.perf_counter() - t0
        assert ei.value.status == _lib.TIMEOUT
    finally:
        assert lib.toposzp_set_test_hold(-1) == _lib.OK
    assert dt < 6.0, f"held call took {dt:.2f} s"
    out = codec.decompress(buf, a.shape).cpu().numpy()
    want = oracle.decompress(buf.cpu().numpy().tobytes(), a.shape)
    assert np.array_equal(out.view(np.uint32), want.view(np.uint32))


def test_batch_decompress_refuses_while_the_hold_is_set():
    """A set hold would be baked into the batch plan's captured graph: the
    batch call refuses instead, and works again once the hold is cleared."""
    from paper_2602_17552_gb300 import batch
    fs = [synth.climate_2d(40, 64, seed=3, device="cuda"), synth.turbulence_3d(16, seed=4, device="cuda")]
    plan = batch.BatchPlan.create(fs, [1e-3, 1e-3], "rel", branches=2)
    plan.compress()
    lib = _lib.load()
    assert lib.toposzp_set_test_hold(0) == _lib.OK
    try:
        with pytest.raises(_lib.TopoSZpError) as ei:
            plan.decompress()
        assert ei.value.status == _lib.INVALID_ARG
    finally:
        assert lib.toposzp_set_test_hold(-1) == _lib.OK
    plan.decompress()
    plan.check()
    for f, it in zip(fs, plan.items):
        want = codec.decompress(codec.compress(f, 1e-3, "rel"), tuple(f.shape))
        assert torch.equal(it.dec.view(torch.int32), want.view(torch.int32))
