"""Served form: every request's result is the same alone and in the mix, and
the mix really overlaps requests on the device."""
import pytest
import torch

from paper_2602_17552_gb300 import serve, synth

pytestmark = pytest.mark.gpu


def _requests(count=14, rate=4000.0, seed=21):
    return synth.request_stream(count=count, rate_hz=rate, seed=seed, min_bytes=64 << 10, max_bytes=6 << 20)


def test_served_results_equal_alone():
    reqs = _requests()
    srv = serve.Server(slots=4, keep_outputs=True)
    stats, outs = srv.run(reqs)
    assert len(outs) == len(reqs)
    for r in reqs:
        alone = serve.plain_result(r)
        assert torch.equal(outs[r.rid], alone), r
    s = stats.summary()
    assert s["requests"] == len(reqs) and stats.max_inflight > 1


def test_serial_mode_same_results():
    reqs = _requests(count=6, seed=22)
    srv = serve.Server(slots=4, keep_outputs=True)
    stats, outs = srv.run(reqs, serial=True)
    assert stats.max_inflight == 1
    for r in reqs:
        assert torch.equal(outs[r.rid], serve.plain_result(r))


def test_admission_waits_for_memory():
    # equal-size compress requests arriving together, with HBM for one at a time
    reqs = [synth.Request(i, 1e-4 * i, "compress",
                          synth.FieldSpec(f"eq{i}", 3, (48, 48, 48), "mixed", 900 + i, "rel", 1e-3, -5 / 3))
            for i in range(6)]
    srv = serve.Server(slots=8, keep_outputs=True)
    srv.budget = serve._bytes_needed(reqs[0].spec.shape(), "compress")
    stats, outs = srv.run(reqs)
    assert stats.max_inflight == 1 and stats.admitted_waits > 0
    for r in reqs:
        assert torch.equal(outs[r.rid], serve.plain_result(r))
