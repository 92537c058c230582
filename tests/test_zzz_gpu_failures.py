"""Failure paths on the GPU without a fault, trap or hang: a bounded device wait
that runs out ends the call with TOPOSZP_ERR_TIMEOUT in its status word, and
the next call on the same context decodes normally."""
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
