"""The allocation-free compress entry point, for callers that cannot hand the
library device memory (an in-situ hook whose device memory belongs to the host
simulation's own pool, or code running while a CUDA graph is being captured).

toposzp_compress_noalloc is called through the C ABI; its stream must equal
the one from toposzp_compress with a caller workspace (bit for bit, the
tolerance every parity test here uses), on two calls in a row, since every call
reuses the same static scratch.  Collected last on purpose, and independent of
the other tests: it passes alone in a fresh process or after them.
"""
import ctypes

import pytest
import torch

from paper_2602_17552_gb300 import _lib, codec, synth

pytestmark = pytest.mark.gpu


def noalloc_compress(field: torch.Tensor, eb: float, mode: str):
    """Call the allocation-free entry point; the output buffers below belong to
    this test (the entry point itself allocates nothing)."""
    L = _lib.load()
    nd, d = codec.field_dims(field.shape)
    out = torch.empty(codec.compress_bound(field.shape), dtype=torch.uint8, device=field.device)
    size = torch.zeros(1, dtype=torch.int64, device=field.device)
    status = torch.full((1,), -1, dtype=torch.int32, device=field.device)
    p = codec.make_params()
    st = L.toposzp_compress_noalloc(field.data_ptr(), nd, _lib.dims3(nd, d),
                                    _lib.EB_REL if mode == "rel" else _lib.EB_ABS, float(eb), ctypes.byref(p),
                                    out.data_ptr(), out.numel(), size.data_ptr(), status.data_ptr(),
                                    int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, int(status.item()), out[:int(size.item())].clone()


@pytest.mark.parametrize("kind", ["2d_max", "3d", "2d_abs"])
def test_noalloc_equals_workspace_entry_point(kind):
    L = _lib.load()
    assert L.toposzp_noalloc_max_points() == 1 << 18
    if kind == "2d_max":
        f, eb, mode = synth.climate_2d(512, 512, seed=11, device="cuda"), 1e-3, "rel"   # exactly the limit
    elif kind == "3d":
        f, eb, mode = synth.turbulence_3d(60, seed=12, device="cuda"), 1e-4, "rel"
    else:
        f = synth.gaussian_bumps_2d(200, 300, count=20, seed=13).cuda()
        eb, mode = 1e-3 * float(f.max() - f.min()), "abs"
    want = codec.compress(f, eb, mode)
    for _ in range(2):   # the shared scratch keeps the previous call's contents
        st, dev_status, got = noalloc_compress(f, eb, mode)
        assert st == _lib.OK and dev_status == 0
        assert torch.equal(got, want)
    # and the stream decodes like the other one
    assert torch.equal(codec.decompress(got, tuple(f.shape)), codec.decompress(want, tuple(f.shape)))


def test_noalloc_rejects_fields_over_the_limit():
    f = torch.zeros((513, 512), dtype=torch.float32, device="cuda")
    st, _, _ = noalloc_compress(f, 1e-3, "rel")
    assert st == _lib.UNSUPPORTED


def test_noalloc_status_split_matches_the_workspace_entry_point():
    """Nonzero dims too large for the library are UNSUPPORTED, as in
    toposzp_compress; zero dims or a bad ndim are INVALID_ARG.  The dims are
    checked on the host before anything touches the (small) buffers."""
    L = _lib.load()
    f = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.empty(4096, dtype=torch.uint8, device="cuda")
    size = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = codec.make_params()
    stream = int(torch.cuda.current_stream().cuda_stream)

    def call(nd, dims):
        d = (ctypes.c_uint64 * 3)(*dims)
        return L.toposzp_compress_noalloc(f.data_ptr(), nd, d, _lib.EB_REL, 1e-3, ctypes.byref(p), out.data_ptr(),
                                          out.numel(), size.data_ptr(), status.data_ptr(), stream)

    assert call(2, (1 << 31, 1, 1)) == _lib.UNSUPPORTED
    assert call(3, (1 << 11, 1 << 10, 1 << 10)) == _lib.UNSUPPORTED
    assert call(2, (0, 5, 1)) == _lib.INVALID_ARG
    assert call(4, (4, 4, 1)) == _lib.INVALID_ARG
    torch.cuda.synchronize()
