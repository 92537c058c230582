"""Host-side bookkeeping of the serving loop (no GPU): the first-fit arena that
admission by free HBM relies on."""
import numpy as np
import pytest

from paper_2602_17552_gb300 import serve


def test_arena_first_fit_alignment_and_coalescing():
    a = serve.Arena(4096, "cpu")
    x = a.alloc(100)            # rounded up to the 256-byte alignment
    y = a.alloc(1000)
    z = a.alloc(256)
    assert x == (0, 256) and y == (256, 1024) and z == (1280, 256)
    assert a.free_bytes == 4096 - 1536
    assert a.alloc(4096) is None                 # does not fit: the request waits
    a.release(*y)
    assert a.alloc(512) == (256, 512)            # first fit reuses the hole
    a.release(*x)
    a.release(256, 512)
    a.release(*z)
    assert a.free == [(0, 4096)]                 # every release coalesced
    assert a.view(512, 256).numel() == 256


def test_arena_never_hands_out_overlapping_ranges():
    import random
    rng = random.Random(3)
    a = serve.Arena(1 << 16, "cpu")
    live = []
    for _ in range(2000):
        if live and rng.random() < 0.45:
            a.release(*live.pop(rng.randrange(len(live))))
        else:
            r = a.alloc(rng.randint(1, 5000))
            if r is not None:
                live.append(r)
        spans = sorted(live)
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2
        assert all(o % 256 == 0 and n % 256 == 0 for o, n in live)
        assert a.free_bytes + sum(n for _, n in live) == 1 << 16


def test_stats_summary_percentiles_and_rate():
    st = serve.ServeStats(latencies_ms=[float(i) for i in range(1, 101)], bytes_total=3_000_000_000, wall_s=1.5,
                          max_inflight=5, admitted_waits=2)
    s = st.summary()
    assert s["requests"] == 100
    assert s["p50_ms"] == pytest.approx(50.5) and s["p99_ms"] == pytest.approx(99.01)
    assert s["mean_ms"] == pytest.approx(50.5)
    assert s["aggregate_gbs"] == pytest.approx(2.0)
    assert (s["max_inflight"], s["memory_waits"]) == (5, 2)
    assert serve.ServeStats().summary()["requests"] == 0     # an empty run reports zeros, not an error


def test_retimed_scales_the_unit_rate_gaps():
    from paper_2602_17552_gb300 import synth
    jobs = [serve.Job(synth.Request(i, 0.0, "compress", None), (4, 4)) for i in range(4)]
    gaps = [0.5, 1.0, 0.25, 2.0]
    at = [j.req.t_arrive for j in serve.retimed(jobs, 2.0, gaps)]
    assert at == pytest.approx([0.25, 0.75, 0.875, 1.875])    # cumulative gaps / rate
    assert [j.req.t_arrive for j in serve.retimed(jobs, float("inf"), gaps)] == [0.0] * 4
    assert [j.req.rid for j in serve.retimed(jobs, 1.0, gaps)] == [0, 1, 2, 3]


def test_admission_size_covers_aligned_workspace_and_output():
    from paper_2602_17552_gb300 import codec
    for shape in ((37, 41), (12, 40, 41)):
        for op in ("compress", "decompress"):
            need = serve._bytes_needed(shape, op)
            ws = codec.compress_workspace_size(shape) if op == "compress" else codec.decompress_workspace_size(shape)
            out = codec.compress_bound(shape) if op == "compress" else 4 * int(np.prod(shape))
            assert need % serve.ALIGN == 0
            assert ws + out <= need < ws + out + 2 * serve.ALIGN
