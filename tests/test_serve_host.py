"""Host-side bookkeeping of the serving loop (no GPU): the first-fit arena that
admission by free HBM relies on."""
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
