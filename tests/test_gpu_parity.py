"""CUDA path against the CPU oracle, element by element.

Bit-exact on everything: the compressed stream (every header field, section
and padding byte), the decompressed float32 values, and the critical-point
labels.  Inputs are seeded synthetic fields; sizes span several 2048-point
tiles with ragged tails, degenerate shapes, and the full workload sizes.
"""
import numpy as np
import pytest
import torch

import oracle
from golden_io import field, load
from paper_2602_17552_gb300 import _lib, codec, synth

pytestmark = pytest.mark.gpu


def section_report(a: bytes, b: bytes) -> str:
    """Name the first differing byte by stream section (for failure messages)."""
    n = min(len(a), len(b))
    diff = next((i for i in range(n) if a[i] != b[i]), n)
    h = oracle.header(b) if len(b) >= 256 else {}
    names = ["off_s1", "off_s2", "off_s4", "off_s6", "off_s5", "off_s7", "total"]
    where = "header"
    for k in names:
        if k in h and diff >= h[k]:
            where = k
    return f"len gpu {len(a)} oracle {len(b)}; first diff at byte {diff} ({where})"


def gpu_roundtrip(a: np.ndarray, eb: float, rel: bool, **kw):
    f = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    buf = codec.compress(f, eb, "rel" if rel else "abs", **kw)
    out = codec.decompress(buf, a.shape)
    return buf.cpu().numpy().tobytes(), out.cpu().numpy()


def assert_parity(a, eb, rel=True, **kw):
    okw = dict(no_topo=kw.get("no_topo", False), rs_sweeps=kw.get("rs_sweeps", 1),
               rbf_k=kw.get("rbf_k", 0), rbf_sigma=kw.get("rbf_sigma", 0.0), rbf_solve=kw.get("rbf_solve", False),
               tile_blocks=kw.get("tile_blocks", False))
    gbuf, gout = gpu_roundtrip(a, eb, rel, **okw)
    obuf = oracle.compress(a, eb, rel=rel, **okw)
    assert gbuf == obuf, section_report(gbuf, obuf)
    oout = oracle.decompress(obuf, a.shape)
    assert np.array_equal(gout.view(np.uint32), oout.view(np.uint32)), \
        f"{np.count_nonzero(gout.view(np.uint32) != oout.view(np.uint32))} decoded values differ"
    return obuf, oout


SMALL = [
    ("bumps256_abs", lambda: synth.gaussian_bumps_2d().numpy(), None),
    ("climate_300x517", lambda: synth.climate_2d(300, 517, seed=2).numpy(), None),
    ("turb_24", lambda: synth.turbulence_3d(24, seed=3).numpy(), None),
    ("mixed3d_45x37x29", lambda: synth.grf((29, 37, 45), -11 / 3, 4).numpy(), None),
    ("adv2d_133x71", lambda: synth.adversarial_small(1, (133, 71)).numpy(), None),
    ("adv3d_17x9x13", lambda: synth.adversarial_small(2, (17, 9, 13)).numpy(), None),
    ("turb_cols_45x32x64", lambda: np.exp(synth.grf((45, 32, 64), -11 / 3, 6).numpy()), None),
]


@pytest.mark.parametrize("name,make,_", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4])
def test_parity_small(name, make, _, eb):
    a = make()
    assert_parity(a, eb, rel=True)


def test_parity_config1_abs_bound():
    """256x256 bumps, absolute bound 1e-3 of the value range."""
    a = synth.gaussian_bumps_2d().numpy()
    eb = 1e-3 * float(a.max() - a.min())
    buf, out = assert_parity(a, eb, rel=False)
    la, lo = oracle.critical_points(a), oracle.critical_points(out)
    e = oracle.topo_errors(la, lo)
    assert e[1].sum() == 0 and e[2].sum() == 0


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (37, 1), (2, 2), (3, 3), (1, 1, 40), (5, 1, 7),
                                   (3, 3, 3), (1, 33), (4, 8, 1), (2, 1025),
                                   # nx % 4 == 0: the vectorised CD path and its boundary rows
                                   (1, 4), (2, 8), (3, 4, 4), (5, 3, 12), (9, 16), (4, 1, 8), (2, 2, 4),
                                   (1, 1, 128), (3, 260),
                                   # planes of whole 128-point chunks: the z-column pass, one and two segments
                                   (5, 8, 16), (40, 16, 32), (70, 4, 64)])
def test_parity_degenerate_shapes(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.integers(-4, 5, size=shape).astype(np.float32) * np.float32(0.25)
    assert_parity(a, 1e-2, rel=True)
    assert_parity(a, 0.3, rel=False)


@pytest.mark.parametrize("shape", [(5, 8, 16), (40, 16, 32), (70, 4, 64), (45, 32, 64), (3, 2, 64)])
def test_parity_column_pass_forced(shape):
    """cd_columns = 1: the z-column pass on fields whose columns are too few
    for the default to take it (4-plane segments, the last one ragged)."""
    from paper_2602_17552_gb300 import autotune
    rng = np.random.default_rng(sum(shape) + 1)
    a = rng.integers(-4, 5, size=shape).astype(np.float32) * np.float32(0.25)
    b = np.exp(synth.grf(shape, -11 / 3, 7).numpy()) if min(shape) > 2 else a
    try:
        autotune.apply({"cd_columns": 1})
        assert_parity(a, 1e-2, rel=True)
        assert_parity(b, 1e-3, rel=True)
    finally:
        autotune.restore()


@pytest.mark.parametrize("shape", [(128, 128, 128), (30, 256, 256)])
def test_parity_column_pass_short_segments(shape):
    """Default tuning on fields with few columns: the column pass with 4-plane
    segments (30 planes: the last segment has 2)."""
    a = np.exp(synth.grf(shape, -11 / 3, 8).numpy())
    assert_parity(a, 1e-3, rel=True)


def test_parity_constant_and_tiny_range():
    assert_parity(np.full((37, 41), -2.5, np.float32), 1e-3, rel=True)
    assert_parity(np.zeros((9, 10, 11), np.float32), 1e-3, rel=True)
    a = np.full((64, 70), 1.0, np.float32)
    a[10, 10] = np.float32(1.001)
    assert_parity(a, 0.01, rel=True)
    # a one-ulp range makes eps ~ 6e-8: too small for M = 1 on both sides
    a[10, 10] = np.nextafter(np.float32(1), np.float32(2))
    with pytest.raises(oracle.OracleError) as eo:
        oracle.compress(a, 0.5, rel=True)
    with pytest.raises(_lib.TopoSZpError) as eg:
        codec.compress(torch.from_numpy(a).cuda(), 0.5, "rel")
    assert eo.value.status == eg.value.status == _lib.EB_TOO_SMALL


@pytest.mark.parametrize("shape", [(50, 60), (12, 16, 20), (6, 8, 16), (40, 4, 64)])
def test_parity_negative_zero_and_denormals(shape):
    """Signed zeros compare equal and subnormal differences keep their sign
    (nx % 4 == 0: the vectorised critical-point pass, 2D and 3D; 128-point
    planes: the z-column pass)."""
    rng = np.random.default_rng(3)
    a = rng.choice(np.array([-0.0, 0.0, 1e-40, -1e-40, 1e-38, -2e-38], np.float32), size=shape)
    assert_parity(a.astype(np.float32), 0.25, rel=True)


@pytest.mark.parametrize("opts", [dict(no_topo=True), dict(rbf_k=3, rbf_sigma=1.0), dict(rbf_k=5),
                                  dict(rbf_k=7, rbf_sigma=0.6), dict(rs_sweeps=3)])
def test_parity_params(opts):
    a = synth.climate_2d(120, 250, seed=9).numpy()
    assert_parity(a, 1e-2, rel=True, **opts)
    b = synth.turbulence_3d(20, seed=5).numpy()
    assert_parity(b, 1e-3, rel=True, **opts)


def test_deterministic_across_calls():
    a = torch.from_numpy(synth.turbulence_3d(32, seed=8).numpy()).cuda()
    outs = [codec.compress(a, 1e-3, "rel").cpu().numpy().tobytes() for _ in range(3)]
    assert outs[0] == outs[1] == outs[2]


@pytest.mark.parametrize("shape", [(256, 256), (90, 333), (12, 40, 41), (1, 77), (33, 44), (6, 7, 12),
                                   (1, 16), (3, 1, 20), (70, 5, 36)])
def test_critical_points_and_topo_errors(shape):
    rng = np.random.default_rng(7)
    a = rng.integers(0, 5, size=shape).astype(np.float32)
    f = torch.from_numpy(a).cuda()
    words, cnt = codec.critical_points(f)
    lab = codec.unpack_labels(words, a.size).cpu().numpy().reshape(shape)
    want = oracle.critical_points(a)
    assert np.array_equal(lab, want)
    assert cnt.cpu().tolist() == [int((want == t).sum()) for t in range(4)]
    b = a + rng.integers(0, 2, size=shape).astype(np.float32)
    wb, _ = codec.critical_points(torch.from_numpy(b).cuda())
    e = codec.topo_errors(words, wb, a.size).cpu().numpy()
    assert np.array_equal(e, oracle.topo_errors(want, oracle.critical_points(b)).astype(np.int64))


def test_device_errors_reported():
    a = synth.gaussian_bumps_2d(40, 50, count=5, seed=2).numpy()
    bad = a.copy()
    bad[3, 4] = np.inf
    with pytest.raises(_lib.TopoSZpError) as ei:
        codec.compress(torch.from_numpy(bad).cuda(), 1e-3, "rel")
    assert ei.value.status == _lib.NONFINITE
    big = (a * 1e6).astype(np.float32)
    with pytest.raises(_lib.TopoSZpError) as ei:
        codec.compress(torch.from_numpy(big).cuda(), 1e-3 * 2 ** -20, "abs")
    assert ei.value.status == _lib.EB_TOO_SMALL
    buf = codec.compress(torch.from_numpy(a).cuda(), 1e-3, "rel")
    for corrupt in (buf[:200].clone(), torch.cat([buf[:100], buf[100:].flip(0)])):
        with pytest.raises(_lib.TopoSZpError) as ei:
            codec.decompress(corrupt, a.shape)
        assert ei.value.status == _lib.CORRUPT_STREAM
    with pytest.raises(_lib.TopoSZpError):
        codec.decompress(buf, (a.shape[0] + 1, a.shape[1]))
    # a damaged payload must never read outside the buffer: widths inflated to 32
    h = oracle.header(buf.cpu().numpy().tobytes())
    dmg = buf.clone()
    dmg[h["off_s2"]:h["off_s2"] + 16] = 32
    with pytest.raises(_lib.TopoSZpError) as ei:
        codec.decompress(dmg, a.shape)
    assert ei.value.status == _lib.CORRUPT_STREAM


def test_device_errors_reported_tile_format():
    """Damaged format-v2 streams come back as CORRUPT_STREAM, with no read
    outside the buffer: a truncated stream, widths inflated to 32 (with and
    without the predictor bit), the predictor bit on a constant block, and a
    format-v1 stream relabelled as version 2 (its block count no longer
    matches the grid's tiles)."""
    a = synth.gaussian_bumps_2d(41, 50, count=5, seed=2).numpy()   # 65 runs of 32, 77 tiles
    f = torch.from_numpy(a).cuda()
    buf = codec.compress(f, 1e-3, "rel", tile_blocks=True)
    h = oracle.header(buf.cpu().numpy().tobytes())
    assert h["version"] == 2
    bad = [buf[:200].clone()]
    for v in (32, 0x80 | 32, 0x80):
        d = buf.clone()
        d[h["off_s2"]:h["off_s2"] + 16] = v
        bad.append(d)
    v1 = codec.compress(f, 1e-3, "rel").clone()
    v1[4] = 2
    bad.append(v1)
    for d in bad:
        with pytest.raises(_lib.TopoSZpError) as ei:
            codec.decompress(d, a.shape)
        assert ei.value.status == _lib.CORRUPT_STREAM
    # the library still decodes a good stream afterwards
    assert torch.equal(codec.decompress(buf, a.shape), codec.decompress(codec.compress(f, 1e-3, "rel"), a.shape))


def test_parity_config2_full():
    """1800 x 3600 climate-like field, relative bounds 1e-2, 1e-3, 1e-4."""
    a = synth.climate_2d(1800, 3600, seed=2, device="cuda").cpu().numpy()
    for eb in (1e-2, 1e-3, 1e-4):
        buf, out = assert_parity(a, eb, rel=True)
        dev = np.abs(a.astype(np.float64) - out).max()
        assert dev <= 2 * oracle.header(buf)["eps"]


@pytest.mark.slow
def test_parity_config3_full():
    """512^3 turbulence-like log-normal field, relative bounds 1e-3 and 1e-5."""
    a = synth.turbulence_3d(512, seed=3, device="cuda").cpu().numpy()
    for eb in (1e-3, 1e-5):
        assert_parity(a, eb, rel=True)


def test_parity_rank_paths_narrow_key_span():
    """A positive field inside [256, 272) (keys span < 2^19), small enough in
    key span for the dense ranks to come from key bitmaps: the stream is the
    oracle's on the bitmap path with the per-bin rank table, on the bitmap path
    without it, and on the radix-sort path.  Which path ran is read from the
    workspace's control block (its first words: min_inv, max_key, nonfinite,
    sort_passes, rank_bitmap, bm_words, bm_off, bin_n)."""
    from paper_2602_17552_gb300 import autotune
    g = synth.grf((96, 96, 96), -11 / 3, 21).numpy()
    a = (264.0 + 7.0 * np.tanh(g / 3.0)).astype(np.float32)
    assert a.min() > 256 and a.max() < 272
    obuf, _ = assert_parity(a, 1e-3, rel=True)
    f = torch.from_numpy(a).cuda()
    ws = torch.empty(codec.compress_workspace_size(a.shape), dtype=torch.uint8, device="cuda")
    seen = {}
    try:
        for mode in (0, 1, -1):
            autotune.apply({**autotune.DEFAULT, "rank_bitmap": mode})
            call = codec.compress_async(f, 1e-3, "rel", ws=ws)
            torch.cuda.synchronize()
            assert int(call.status.item()) == 0
            got = call.out[: int(call.size.item())].cpu().numpy().tobytes()
            ctrl = ws[:32].cpu().numpy().view(np.uint32)
            seen[mode] = (int(ctrl[4]), int(ctrl[7]))
            assert got == obuf, f"rank_bitmap={mode}: " + section_report(got, obuf)
    finally:
        autotune.restore()
    assert seen[0][0] == 1 and seen[0][1] > 0, seen     # bitmaps + bin table
    assert seen[1][0] == 1 and seen[1][1] == 0, seen    # bitmaps, no table
    assert seen[-1][0] == 0, seen                      # radix sort


@pytest.mark.parametrize("shape", [(96, 96, 96), (600, 700)])
def test_parity_saddle_rounds_many_tiles(shape):
    """RS^ rounds on a field of many decode tiles (RBF radius 3, two sweeps):
    with neighbourhood records and with direct field reads, the oracle's field."""
    from paper_2602_17552_gb300 import autotune
    if len(shape) == 3:
        a = synth.turbulence_3d(shape[0], seed=11).numpy()
    else:
        a = synth.climate_2d(*shape, seed=11).numpy()
    opts = dict(rbf_k=7, rs_sweeps=2)
    obuf = oracle.compress(a, 1e-3, rel=True, **opts)
    oout = oracle.decompress(obuf, a.shape)
    f = torch.from_numpy(a).cuda()
    try:
        for cfg in ({}, {"saddle_records": -1}):
            autotune.apply({**autotune.DEFAULT, **cfg})
            buf = codec.compress(f, 1e-3, "rel", **opts)
            assert buf.cpu().numpy().tobytes() == obuf, cfg
            out = codec.decompress(buf, a.shape).cpu().numpy()
            assert np.array_equal(out.view(np.uint32), oout.view(np.uint32)), \
                (cfg, int(np.count_nonzero(out.view(np.uint32) != oout.view(np.uint32))))
    finally:
        autotune.restore()


@pytest.mark.parametrize("shape", [(33, 65), (9, 10, 11), (100, 300), (20, 30, 40)])
def test_parity_every_point_an_extremum(shape):
    """A checkerboard of random magnitudes: every point is a minimum or a
    maximum (the largest extremum lists and rank stream a field can have)."""
    rng = np.random.default_rng(5)
    parity = np.indices(shape).sum(axis=0) % 2
    a = ((1.0 + rng.random(shape)) * np.where(parity == 0, 1.0, -1.0)).astype(np.float32)
    for eb in (1e-5, 1e-2):
        assert_parity(a, eb, rel=True)


@pytest.mark.parametrize("name", ["h4_saddle.txt", "rs_shepard_2d_k5.txt", "rs_shepard_2d_k5_edge.txt",
                                  "rs_clamp_3d_k3.txt", "rs_reject_new_type_3d.txt"])
def test_parity_rs_hand_cases(name):
    """The hand-worked RS^ fixtures (Section IV-B(3)): the kernel value with
    r = 2, the cut ball at the boundary, the 3D clamp, and the refusal of a
    correction that would create a new critical point."""
    g = load(name)
    k = int(g.get("rbf_k", 3))
    s = float(g.get("rbf_sigma", 1.0))
    assert_parity(field(g), float(g["eps"]), rel=False, rbf_k=k, rbf_sigma=s)


@pytest.mark.parametrize("k", [3, 5, 7])
@pytest.mark.parametrize("name,make", [
    ("climate_120x250", lambda: synth.climate_2d(120, 250, seed=9).numpy()),
    ("turb_20", lambda: synth.turbulence_3d(20, seed=5).numpy()),
    ("adv3d_17x9x13", lambda: synth.adversarial_small(2, (17, 9, 13)).numpy()),
    ("mixed3d_45x37x29", lambda: synth.grf((29, 37, 45), -11 / 3, 4).numpy()),
], ids=["climate_120x250", "turb_20", "adv3d_17x9x13", "mixed3d_45x37x29"])
def test_parity_rbf_solve(name, make, k):
    """The literal RBF interpolation (Section IV-B(3), Eqs. RBF-interp-final
    and RBF-eval; header flag RBF_SOLVE): the weights solved on the device in
    binary64 (up to 122 nodes at r = 3 in 3D) and the unclamped refinement
    give the oracle's stream and field bit for bit."""
    a = make()
    for eb in (1e-2, 1e-3):
        assert_parity(a, eb, rel=True, rbf_solve=True, rbf_k=k, rbf_sigma=0.5 + 0.1 * k / 2)


@pytest.mark.parametrize("shape", [(96, 96, 96), (600, 700)])
def test_parity_rbf_solve_many_tiles(shape):
    """Literal interpolation on fields of many decode tiles, adaptive kernel,
    two sweeps: with neighbourhood records and with direct field reads."""
    from paper_2602_17552_gb300 import autotune
    a = synth.turbulence_3d(shape[0], seed=11).numpy() if len(shape) == 3 else \
        synth.climate_2d(*shape, seed=11).numpy()
    opts = dict(rbf_solve=True, rs_sweeps=2)
    obuf = oracle.compress(a, 1e-3, rel=True, **opts)
    oout = oracle.decompress(obuf, a.shape)
    f = torch.from_numpy(a).cuda()
    try:
        for cfg in ({}, {"saddle_records": -1}, {"dec_split": 1}):
            autotune.apply({**autotune.DEFAULT, **cfg})
            buf = codec.compress(f, 1e-3, "rel", **opts)
            assert buf.cpu().numpy().tobytes() == obuf, cfg
            out = codec.decompress(buf, a.shape).cpu().numpy()
            assert np.array_equal(out.view(np.uint32), oout.view(np.uint32)), \
                (cfg, int(np.count_nonzero(out.view(np.uint32) != oout.view(np.uint32))))
    finally:
        autotune.restore()


def test_parity_rbf_solve_hand_cases():
    """The hand-worked RS^ fixtures decoded with the literal interpolation."""
    for name in ("h4_saddle.txt", "rs_shepard_2d_k5.txt", "rs_shepard_2d_k5_edge.txt", "rs_clamp_3d_k3.txt",
                 "rs_reject_new_type_3d.txt"):
        g = load(name)
        assert_parity(field(g), float(g["eps"]), rel=False, rbf_k=int(g.get("rbf_k", 3)),
                      rbf_sigma=float(g.get("rbf_sigma", 1.0)), rbf_solve=True)


def _tile_field(shape, seed=4):
    if len(shape) == 3 and min(shape) >= 8:
        return synth.grf(shape, -11 / 3, seed).numpy()
    if len(shape) == 2 and min(shape) >= 8:
        return synth.climate_2d(*shape, seed=seed).numpy()
    return np.random.default_rng(seed).standard_normal(shape).astype(np.float32)


@pytest.mark.parametrize("shape", [(300, 517), (24, 24, 24), (29, 37, 45), (33, 65), (9, 10, 11), (1, 1), (1, 37),
                                   (37, 1), (1, 1, 40), (5, 1, 7), (40, 1, 1), (2, 3, 5), (7, 9, 13)],
                         ids=lambda s: "x".join(map(str, s)))
def test_parity_tile_blocks(shape):
    """Format v2, tile-shaped blocks (TOPOSZP_TILE_BLOCKS): the CUDA stream
    equals the oracle's byte for byte (the per-block predictor choice and
    the clamped codes of blocks that stick out of the grid included), and
    the decoded field equals both the oracle's and the format-v1 field."""
    a = _tile_field(shape)
    for eb, nt in ((1e-2, False), (1e-4, False), (1e-3, True)):
        _, oout = assert_parity(a, eb, rel=True, no_topo=nt, tile_blocks=True)
        _, v1 = gpu_roundtrip(a, eb, True, no_topo=nt)
        assert np.array_equal(oout.view(np.uint32), v1.view(np.uint32))


@pytest.mark.parametrize("shape", [(96, 96, 96), (600, 700)])
def test_parity_tile_blocks_many_tiles(shape):
    """Format v2 on fields of many tiles, through the fused decoder (S1 done
    by the tile kernel) with and without neighbourhood records, and through
    the split stages."""
    from paper_2602_17552_gb300 import autotune
    a = synth.turbulence_3d(shape[0], seed=11).numpy() if len(shape) == 3 else \
        synth.climate_2d(*shape, seed=11).numpy()
    obuf = oracle.compress(a, 1e-3, rel=True, tile_blocks=True)
    oout = oracle.decompress(obuf, a.shape)
    f = torch.from_numpy(a).cuda()
    try:
        for cfg in ({}, {"saddle_records": -1}, {"dec_split": 1}):
            autotune.apply({**autotune.DEFAULT, **cfg})
            buf = codec.compress(f, 1e-3, "rel", tile_blocks=True)
            assert buf.cpu().numpy().tobytes() == obuf, cfg
            out = codec.decompress(buf, a.shape).cpu().numpy()
            assert np.array_equal(out.view(np.uint32), oout.view(np.uint32)), cfg
    finally:
        autotune.restore()
    info = codec.inspect(buf)
    assert info.flags & _lib.TILE_BLOCKS
