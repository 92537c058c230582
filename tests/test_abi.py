"""The C-ABI library builds, loads, exports every symbol include/toposzp.h
declares, and its host-only functions behave (no GPU needed: none of these
calls reaches a CUDA API)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2602_17552_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "toposzp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(toposzp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_exports(lib):
    names = declared_symbols()
    assert set(names) == set(_lib.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings_and_defaults(lib):
    for code in range(9):
        s = lib.toposzp_status_string(code)
        assert s and s != b"unknown status"
    p = _lib.Params()
    lib.toposzp_default_params(ctypes.byref(p))
    assert (p.flags, p.rs_sweeps, p.rbf_k, p.rbf_sigma) == (0, 1, 0, 0.0)


@pytest.mark.parametrize("shape", [(256, 256), (1800, 3600), (1, 1), (1, 37), (7, 9, 11), (3, 1, 5)])
def test_bounds_cover_the_oracle_stream(lib, shape):
    nd = len(shape)
    dims = _lib.dims3(nd, tuple(reversed(shape)))
    bound = lib.toposzp_compress_bound(nd, dims)
    assert bound >= 256
    if np.prod(shape) <= 4096:
        rng = np.random.default_rng(0)
        a = rng.normal(size=shape).astype(np.float32)
        assert len(oracle.compress(a, 1e-4, rel=True)) <= bound
    assert lib.toposzp_compress_workspace_size(nd, dims) > 0
    assert lib.toposzp_decompress_workspace_size(nd, dims) > 0


def test_invalid_arguments_rejected_on_host(lib):
    dims = _lib.dims3(2, (8, 8))
    p = _lib.Params()
    lib.toposzp_default_params(ctypes.byref(p))
    fake = ctypes.c_void_p(256)   # never dereferenced: checks fail first
    assert lib.toposzp_compress(None, 2, dims, 1, 1e-3, ctypes.byref(p), fake, 1 << 20, fake, fake,
                                1 << 20, fake, None) == _lib.INVALID_ARG
    assert lib.toposzp_compress(fake, 4, dims, 1, 1e-3, ctypes.byref(p), fake, 1 << 20, fake, fake,
                                1 << 20, fake, None) == _lib.INVALID_ARG
    assert lib.toposzp_compress(fake, 2, dims, 1, -1.0, ctypes.byref(p), fake, 1 << 20, fake, fake,
                                1 << 20, fake, None) == _lib.INVALID_ARG
    assert lib.toposzp_compress(fake, 2, dims, 1, 1e-3, ctypes.byref(p), fake, 10, fake, fake,
                                1 << 20, fake, None) == _lib.BUFFER_TOO_SMALL
    assert lib.toposzp_compress(fake, 2, dims, 1, 1e-3, ctypes.byref(p), fake, 1 << 20, fake, fake,
                                16, fake, None) == _lib.BUFFER_TOO_SMALL
    big = _lib.dims3(3, (2048, 2048, 1024))
    assert lib.toposzp_compress(fake, 3, big, 1, 1e-3, ctypes.byref(p), fake, 1 << 20, fake, fake,
                                1 << 20, fake, None) == _lib.UNSUPPORTED
    p.rbf_k = 4
    assert lib.toposzp_compress(fake, 2, dims, 1, 1e-3, ctypes.byref(p), fake, 1 << 20, fake, fake,
                                1 << 20, fake, None) == _lib.INVALID_ARG
    assert lib.toposzp_decompress(fake, 100, fake, 0, fake, 1 << 20, fake, None) == _lib.INVALID_ARG


def test_inspect_reads_oracle_header(lib):
    a = np.random.default_rng(1).normal(size=(6, 10, 12)).astype(np.float32)
    buf = oracle.compress(a, 1e-3, rel=True)
    info = _lib.Info()
    cbuf = ctypes.create_string_buffer(buf[:256], 256)
    assert lib.toposzp_inspect(cbuf, 256, ctypes.byref(info)) == 0
    h = oracle.header(buf)
    assert info.ndim == 3 and list(info.dims) == [12, 10, 6] and info.n == a.size
    assert info.total_size == len(buf) and info.k_min == h["k_min"] and info.k_max == h["k_max"]
    bad = ctypes.create_string_buffer(b"XXXX" + buf[4:256], 256)
    assert lib.toposzp_inspect(bad, 256, ctypes.byref(info)) == _lib.CORRUPT_STREAM


@pytest.mark.parametrize("shape", [(33, 65), (9, 10, 11)])
def test_bound_covers_the_worst_case_stream(lib, shape):
    """Every point an extremum (a checkerboard of random magnitudes: each face
    neighbour has the other sign) and wide residuals (a tight bound): the rank
    stream and the payload are as large as they get, still within the bound."""
    rng = np.random.default_rng(5)
    parity = np.indices(shape).sum(axis=0) % 2
    a = ((1.0 + rng.random(shape)) * np.where(parity == 0, 1.0, -1.0)).astype(np.float32)
    buf = oracle.compress(a, 1e-5, rel=True)
    h = oracle.header(buf)
    assert h["k_min"] + h["k_max"] == a.size
    nd = len(shape)
    assert len(buf) <= lib.toposzp_compress_bound(nd, _lib.dims3(nd, tuple(reversed(shape))))


def test_size_limits_on_host(lib):
    """Fields of up to 2^31 - 1 points are sized; 2^31 points are not; a zero
    extent is an invalid argument (all decided on the host)."""
    largest, too_big = _lib.dims3(2, (2 ** 31 - 1, 1)), _lib.dims3(2, (2 ** 16, 2 ** 15))
    for f in (lib.toposzp_compress_bound, lib.toposzp_compress_workspace_size,
              lib.toposzp_decompress_workspace_size, lib.toposzp_workspace_size):
        assert f(2, largest) > 0
        assert f(2, too_big) == 0
    p = _lib.Params()
    lib.toposzp_default_params(ctypes.byref(p))
    fake = ctypes.c_void_p(256)
    for dims in ((0, 8), (8, 0)):
        assert lib.toposzp_compress(fake, 2, _lib.dims3(2, dims), 1, 1e-3, ctypes.byref(p), fake, 1 << 20, fake,
                                    fake, 1 << 20, fake, None) == _lib.INVALID_ARG
    assert lib.toposzp_compress(fake, 2, too_big, 1, 1e-3, ctypes.byref(p), fake, 1 << 20, fake, fake,
                                1 << 20, fake, None) == _lib.UNSUPPORTED


def test_test_hold_arguments(lib):
    assert lib.toposzp_set_test_hold(-2) == _lib.INVALID_ARG
    assert lib.toposzp_set_test_hold(3) == _lib.OK
    assert lib.toposzp_set_test_hold(-1) == _lib.OK


@pytest.mark.parametrize("offset,value", [
    (40, 4), (96, 0), (96, 17), (64, 0x7F800000), (72, 0xBF800000), (88, 4), (112, 1),
    (120, 10 ** 6), (160, 0), (192, 7), (200, 1 << 40),
])
def test_inspect_refuses_what_the_oracle_refuses(lib, offset, value):
    """The host header parser holds every field to the range compression writes,
    like the oracle's decoder: each damaged header is CORRUPT_STREAM for both."""
    import struct
    a = np.random.default_rng(2).normal(size=(20, 24)).astype(np.float32)
    buf = bytearray(oracle.compress(a, 1e-3, rel=True))
    width = 8 if offset in (112, 120, 160, 192, 200) else 4
    buf[offset:offset + width] = struct.pack("<Q" if width == 8 else "<I", value)
    info = _lib.Info()
    cbuf = ctypes.create_string_buffer(bytes(buf[:256]), 256)
    assert lib.toposzp_inspect(cbuf, 256, ctypes.byref(info)) == _lib.CORRUPT_STREAM
    with pytest.raises(oracle.OracleError):
        oracle.decompress(bytes(buf), a.shape)


@pytest.mark.parametrize("shape,opts", [((6, 10, 12), {}), ((33, 65), {"no_topo": True}), ((1, 1), {}),
                                        ((9, 10, 11), {"rbf_k": 7, "rs_sweeps": 16})])
def test_inspect_accepts_every_oracle_header(lib, shape, opts):
    a = np.random.default_rng(4).normal(size=shape).astype(np.float32)
    buf = oracle.compress(a, 1e-3, rel=True, **opts)
    info = _lib.Info()
    cbuf = ctypes.create_string_buffer(buf[:256], 256)
    assert lib.toposzp_inspect(cbuf, 256, ctypes.byref(info)) == _lib.OK
    assert info.total_size == len(buf)


def test_tuning_classes_on_host(lib):
    """Launch geometry per (ndim, size class): the class of a shape, a class
    setting taking over from the default, clearing it, and refused values."""
    import ctypes
    from paper_2602_17552_gb300 import _lib
    d = lambda *x: (ctypes.c_uint64 * 3)(*(list(x) + [1] * (3 - len(x))))
    assert [lib.toposzp_tuning_class(2, d(a, b)) for a, b in ((255, 256), (256, 256), (1024, 1024), (4096, 4096))] \
        == [0, 1, 2, 3]
    assert lib.toposzp_tuning_class(3, d(0, 4, 4)) == -1
    t = _lib.Tuning()
    base = _lib.Tuning()
    assert lib.toposzp_get_tuning(3, d(128, 128, 128), ctypes.byref(base)) == _lib.OK
    try:
        t.cd_threads, t.cd_blocks_per_sm, t.dec_split, t.launch_overlap = 512, 4, 1, -1
        assert lib.toposzp_set_tuning_class(3, 2, ctypes.byref(t)) == _lib.OK
        got = _lib.Tuning()
        assert lib.toposzp_get_tuning(3, d(128, 128, 128), ctypes.byref(got)) == _lib.OK
        assert (got.cd_threads, got.cd_blocks_per_sm, got.dec_split, got.launch_overlap) == (512, 4, 1, -1)
        assert lib.toposzp_get_tuning(2, d(2000, 2000), ctypes.byref(got)) == _lib.OK   # the 2D row is untouched
        assert lib.toposzp_set_tuning_class(3, 2, None) == _lib.OK
        assert lib.toposzp_get_tuning(3, d(128, 128, 128), ctypes.byref(got)) == _lib.OK
        assert got.cd_threads != 512 or base.cd_threads == 512
        t.launch_overlap = 1
        assert lib.toposzp_set_tuning_class(3, 1, ctypes.byref(t)) == _lib.INVALID_ARG
        t.launch_overlap, t.cd_threads = 0, 100
        assert lib.toposzp_set_tuning_class(3, 1, ctypes.byref(t)) == _lib.INVALID_ARG
        assert lib.toposzp_set_tuning_class(4, 1, None) == _lib.INVALID_ARG
        assert lib.toposzp_set_tuning_class(2, 4, None) == _lib.INVALID_ARG
    finally:
        _lib.apply_tuning_file(lib)
