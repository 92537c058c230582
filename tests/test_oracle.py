"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-worked
fixtures from the paper's examples (tests/golden), exact rational arithmetic,
brute-force enumeration written from the paper's definitions, a library routine
(scipy's dense ranking), symmetry invariants, and the properties the paper
proves or reports (no FP / FT, relaxed bound).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_io import field, grid, ints, load
from paper_2602_17552_gb300 import synth

R, MIN, SAD, MAX = 0, 1, 2, 3


# ------------------------------------------------------------------ helpers

def header_q(buf):
    h = oracle.header(buf)
    return h, np.float32(h["w_f"]), np.float32(h["h_f"])


def bin_codes(a, buf):
    """Codes from the stream's own constants, computed here in float32 numpy:
    q = floor(fl(fl(a * r) + 0.5)) (Section II-C round-half-up)."""
    h = oracle.header(buf)
    r = np.float32(h["r_f"])
    x = (np.asarray(a, np.float32) * r).astype(np.float32)
    y = (x + np.float32(0.5)).astype(np.float32)
    return np.floor(y).astype(np.int64)


def brute_labels_2d(a):
    """Section IV-A(1) written out with the paper's t/d/l/r names; corners use two
    neighbours, edges three; a saddle needs all four."""
    ny, nx = a.shape
    out = np.zeros(a.shape, np.uint8)
    for y in range(ny):
        for x in range(nx):
            p = a[y, x]
            t = a[y - 1, x] if y > 0 else None
            d = a[y + 1, x] if y + 1 < ny else None
            l = a[y, x - 1] if x > 0 else None
            r = a[y, x + 1] if x + 1 < nx else None
            avail = [v for v in (t, d, l, r) if v is not None]
            if not avail:
                continue
            if all(p < v for v in avail):
                out[y, x] = MIN
            elif all(p > v for v in avail):
                out[y, x] = MAX
            elif None not in (t, d, l, r) and (
                    (p < t and p < d and p > l and p > r) or (p > t and p > d and p < l and p < r)):
                out[y, x] = SAD
    return out


# ----------------------------------------------------------- QZ (Section II-C)

def test_fig2_bins_and_lost_maximum():
    g = load("fig2_lost_max.txt")
    a = grid(g["field"], np.float32).astype(np.float32)
    eps = float(g["eps"])
    buf = oracle.compress(a, eps, rel=False)
    assert (bin_codes(a, buf) == grid(g["bins"], int)).all()
    p = oracle.qparams(a, False, eps)
    assert (oracle.quantize(a, p).reshape(a.shape) == grid(g["bins"], int)).all()
    assert (oracle.critical_points(a) == grid(g["labels"], int)).all()
    out, d0, d1, stats = oracle.decompress(buf, a.shape, stages=True)
    # QZ^ alone loses the maximum (Fig. 2) ...
    assert (oracle.critical_points(d0) == grid(g["labels_d0"], int)).all()
    # ... and the maxima stencil restores it to max_nbr + 1 ulp
    w = np.float32(oracle.header(buf)["w_f"])
    assert d0[1, 1] == w
    assert out[1, 1] == np.nextafter(w, np.float32(np.inf))
    assert (oracle.critical_points(out) == grid(g["labels"], int)).all()
    assert abs(float(out[1, 1]) - float(a[1, 1])) <= eps


def test_quantizer_is_round_half_up_of_exact_quotient():
    """q equals floor(a / w + 1/2) in exact rational arithmetic, except within the
    binary32 rounding distance of a bin boundary."""
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.normal(0, 3, 4000), rng.uniform(-1e3, 1e3, 2000)]).astype(np.float32)
    for eps in (1e-3, 0.37, 2.5):
        p = oracle.qparams(a, False, eps)
        q = oracle.quantize(a, p)
        w = Fraction(float(np.float32(p.w_f)))
        checked = 0
        for v, qq in zip(a.tolist(), q.tolist()):
            t = Fraction(v) / w + Fraction(1, 2)
            fl = math.floor(t)
            tol = abs(float(t)) * 2.0 ** -22 + 2.0 ** -20   # binary32 rounding of a*r and +0.5
            if float(t - fl) < tol or 1 - float(t - fl) < tol:
                continue        # within rounding distance of a boundary
            assert qq == fl
            checked += 1
        assert checked > 5000


@pytest.mark.parametrize("scale", [1.0, 1e3, 1e-6])
def test_pointwise_bound_exact(scale):
    """|a - QZ^(QZ(a))| <= eps checked in exact rationals, including values just
    either side of every bin boundary and the largest |a| the bound admits."""
    rng = np.random.default_rng(5)
    eps = 1e-3 * scale
    base = rng.uniform(-1, 1, 3000) * scale
    edges = (np.arange(-50, 50) + 0.5) * 2 * eps
    near = np.concatenate([edges, np.nextafter(edges.astype(np.float32), np.float32(np.inf)),
                           np.nextafter(edges.astype(np.float32), np.float32(-np.inf))])
    big = np.array([eps * 2 ** 19.9, -eps * 2 ** 19.9])
    a = np.concatenate([base, near, big]).astype(np.float32)
    p = oracle.qparams(a, False, eps)
    assert p.h_f <= eps and p.h_f >= eps / 2
    q = oracle.quantize(a, p)
    ah = oracle.dequantize(q, p)
    e = Fraction(eps)
    for v, r in zip(a.tolist(), ah.tolist()):
        assert abs(Fraction(v) - Fraction(r)) <= e


def test_quantizer_monotone():
    """Section III-B relies on a1 < a2 => a^1 <= a^2; checked on sorted floats."""
    rng = np.random.default_rng(3)
    a = np.sort(np.concatenate([rng.normal(0, 10, 20000),
                                np.linspace(-1, 1, 5001)]).astype(np.float32))
    for eps in (1e-4, 3e-3, 0.1):
        p = oracle.qparams(a, False, eps)
        q = oracle.quantize(a, p)
        ah = oracle.dequantize(q, p)
        assert (np.diff(q) >= 0).all()
        assert (np.diff(ah) >= 0).all()


def test_eb_too_small_and_constant_field():
    a = np.linspace(0, 1e3, 64, dtype=np.float32).reshape(8, 8)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.compress(a, 1e3 * 2 ** -21, rel=False)
    assert ei.value.status == oracle.EB_TOO_SMALL
    c = np.full((5, 7), -3.25, np.float32)
    buf = oracle.compress(c, 1e-3, rel=True)        # eps = 0 on a constant field
    assert (oracle.decompress(buf, c.shape) == c).all()
    bad = a.copy()
    bad[2, 3] = np.nan
    with pytest.raises(oracle.OracleError) as ei:
        oracle.compress(bad, 1e-2, rel=True)
    assert ei.value.status == oracle.NONFINITE


# --------------------------------------------------------- CD (Section IV-A(1))

def test_cd_hand_3x3():
    g = load("h3_cd_3x3.txt")
    a = grid(g["field"], np.float32).astype(np.float32)
    assert (oracle.critical_points(a) == grid(g["labels"], int)).all()


def test_cd_hand_3x3x3():
    g = load("h3d_cd_3x3x3.txt")
    a = np.zeros((3, 3, 3), np.float32)          # [z, y, x]
    for z, y, x in itertools.product(range(3), repeat=3):
        odd = (x == 1) + (y == 1) + (z == 1)
        if odd == 3:
            a[z, y, x] = 5
        elif odd == 2:                           # face centre: the axis not at 1
            a[z, y, x] = 9 if x != 1 else (1 if y != 1 else 2)
        elif odd == 1:
            a[z, y, x] = 3
    want = np.stack([grid(g[f"labels_z{z}"], int) for z in range(3)])
    assert (oracle.critical_points(a) == want).all()


def test_cd_brute_force_all_3x3_over_three_values():
    """Every 3x3 grid over {0,1,2} (3^9 of them) against the paper's 2D rule."""
    vals = np.array(list(itertools.product((0.0, 1.0, 2.0), repeat=9)), np.float32)
    for v in vals:
        a = v.reshape(3, 3)
        assert (oracle.critical_points(a) == brute_labels_2d(a)).all()


@pytest.mark.parametrize("shape", [(5, 5), (4, 7), (1, 9), (9, 1), (1, 1), (2, 2), (6, 5)])
def test_cd_brute_force_random(shape):
    rng = np.random.default_rng(sum(shape))
    for _ in range(40):
        a = rng.integers(0, 4, size=shape).astype(np.float32)
        assert (oracle.critical_points(a) == brute_labels_2d(a)).all()


def test_cd_symmetries_3d():
    """Axis permutations permute the labels; negation swaps m and M; a positive
    affine map changes nothing -- catches stride, index and sign slips."""
    rng = np.random.default_rng(9)
    swap = np.array([R, MAX, SAD, MIN], np.uint8)
    for shape in [(4, 5, 6), (3, 3, 7), (1, 4, 4)]:
        a = rng.integers(0, 5, size=shape).astype(np.float32)
        lab = oracle.critical_points(a)
        for perm in itertools.permutations(range(3)):
            b = np.ascontiguousarray(a.transpose(perm))
            assert (oracle.critical_points(b) == lab.transpose(perm)).all()
        assert (oracle.critical_points(-a) == swap[lab]).all()
        assert (oracle.critical_points(3 * a + 7) == lab).all()
    # 2D transpose
    a = rng.normal(size=(13, 17)).astype(np.float32)
    assert (oracle.critical_points(np.ascontiguousarray(a.T)) == oracle.critical_points(a).T).all()


def test_no_adjacent_strict_maxima():
    a = synth.adversarial_small(4, (16, 12, 5)).numpy()
    lab = oracle.critical_points(a)
    for ax in range(3):
        m = lab == MAX
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = slice(0, -1)
        sl1[ax] = slice(1, None)
        assert not (m[tuple(sl0)] & m[tuple(sl1)]).any()


# ----------------------------------------------------------- RP (IV-A(2))

def test_fig5_ranks_and_restored_order():
    g = load("fig5_rank_order.txt")
    a = grid(g["field"], np.float32).astype(np.float32)
    eps = float(g["eps"])
    lab = oracle.critical_points(a)
    assert (lab == grid(g["labels"], int)).all()
    p = oracle.qparams(a, False, eps)
    assert list(oracle.ranks(a, lab, p)) == ints(g["delta_seq"])
    out = oracle.decompress(oracle.compress(a, eps, rel=False), a.shape)
    m1, m2 = out[1, 1], out[1, 5]
    assert m1 < m2                                # M1 < M2 restored (Fig. 5)
    assert (oracle.critical_points(out) == lab).all()


def test_ranks_match_scipy_dense_rank_per_bin():
    """RP equals scipy's dense ranking inside each (type, bin) group; maxima
    ranked upward, minima downward."""
    from scipy.stats import rankdata
    a = synth.adversarial_small(7, (40, 30)).numpy()
    a = a + np.float32(0.01) * synth.gaussian_bumps_2d(30, 40, count=6, seed=2).numpy()
    a = a.astype(np.float32)
    lab = oracle.critical_points(a)
    p = oracle.qparams(a, True, 2e-2)
    delta = oracle.ranks(a, lab, p)
    flat, lf = a.ravel(), lab.ravel()
    q = oracle.quantize(flat, p)
    want = {}
    for t in (MIN, MAX):
        for b in np.unique(q[lf == t]):
            idx = np.nonzero((lf == t) & (q == b))[0]
            vals = flat[idx] if t == MAX else -flat[idx]
            for i, rk in zip(idx, rankdata(vals, method="dense")):
                want[i] = int(rk)
    seq = [want[i] for i in np.nonzero((lf == MIN) | (lf == MAX))[0]]
    assert list(delta) == seq
    assert delta.min() >= 1 and (delta > 1).any()


# ------------------------------------------------ B + LZ + BE (II-C, IV-A)

def test_codec_hand_block():
    g = load("codec_block.txt")
    codes = np.array(ints(g["codes"]), np.float32).reshape(1, -1)
    buf = oracle.compress(codes, float(g["eps"]), rel=False)
    h = oracle.header(buf)
    b = np.frombuffer(buf, np.uint8)
    u32 = lambda off, cnt: np.frombuffer(b[off:off + 4 * cnt].tobytes(), "<u4")
    assert u32(h["off_s1"], 1)[0] == int(g["const_bitmap_word0"], 0)
    assert list(b[h["off_s2"]:h["off_s2"] + 2]) == ints(g["widths"])
    assert list(np.frombuffer(b[h["off_s4"]:h["off_s4"] + 8].tobytes(), "<i4")) == ints(g["firsts"])
    assert list(u32(h["off_s5"], h["pay_words"])) == ints(g["payload"])
    assert u32(h["off_s6"], 1)[0] == int(g["labels_word0"], 0)
    assert h["k_min"] == 1 and h["k_max"] == 1
    # rank stream: one constant block with first value 1
    s7 = h["off_s7"]
    assert u32(s7, 1)[0] == 1
    w = np.float32(h["w_f"])
    assert (oracle.decompress(buf, codes.shape) == (codes * w).astype(np.float32)).all()


def _expected_size(q, n, topo, k_delta):
    """Closed-form stream size from the per-block widths (Section IV-A layout)."""
    def a16(x):
        return (x + 15) // 16 * 16

    def blocks(seq):
        nb = -(-len(seq) // 32)
        pad = np.concatenate([seq, np.repeat(seq[-1:], nb * 32 - len(seq))]) if len(seq) else seq
        words = 0
        for b in range(nb):
            blk = pad[b * 32:(b + 1) * 32].astype(np.int64)
            d = np.abs(np.diff(blk))
            w = int(d.max()).bit_length() if d.size else 0
            words += (1 + w) if w else 0
        return nb, words
    nb, words = blocks(q)
    off = a16(256 + 4 * (-(-nb // 32)))
    off = a16(off + nb)
    off = a16(off + 4 * nb)
    off = a16(off + (4 * (-(-n // 16)) if topo else 0))
    end = off + 4 * words
    if topo:
        nbd, rw = blocks(k_delta)
        off = a16(end)
        off = a16(off + 4 * (-(-nbd // 32)))
        off = a16(off + nbd)
        off = a16(off + 4 * nbd)
        end = off + 4 * rw
    return end


@pytest.mark.parametrize("n", [1, 31, 32, 33, 64, 65, 1000])
def test_codec_roundtrip_and_size_adversarial(n):
    rng = np.random.default_rng(n)
    seqs = [np.zeros(n), np.full(n, 7.0),
            (np.arange(n) % 2) * 2.0 ** 18 - 2.0 ** 17,
            rng.integers(-2 ** 18, 2 ** 18, n).astype(np.float64),
            np.cumsum(rng.integers(-3, 4, n)).astype(np.float64)]
    for s in seqs:
        a = s.astype(np.float32).reshape(1, n)
        buf = oracle.compress(a, 0.5, rel=False, no_topo=True)
        out = oracle.decompress(buf, a.shape)
        q = bin_codes(a, buf).ravel()
        if s.min() != s.max() and np.abs(s).max() < 2 ** 16:
            assert (q == s).all()                        # codes equal the integers at eps = 0.5
        w = np.float32(oracle.header(buf)["w_f"])
        assert (out.ravel() == (q.astype(np.float32) * w).astype(np.float32)).all()
        assert len(buf) == _expected_size(q, n, False, None)


def test_stream_size_closed_form_with_topology():
    a = synth.gaussian_bumps_2d(45, 70, count=12, seed=4).numpy()
    buf = oracle.compress(a, 1e-3, rel=True)
    lab = oracle.critical_points(a)
    p = oracle.qparams(a, True, 1e-3)
    delta = oracle.ranks(a, lab, p)
    q = bin_codes(a, buf).ravel()
    assert len(buf) == _expected_size(q, a.size, True, delta)
    h = oracle.header(buf)
    # Section IV-A stream order: const info, block metadata, first elements,
    # labels (fixed-size sections), then sign+magnitude planes, then ranks
    offs = [h[k] for k in ("off_s1", "off_s2", "off_s4", "off_s6", "off_s5", "off_s7")]
    assert offs == sorted(offs) and all(o % 16 == 0 for o in offs)


# -------------------------------------------------- decompression (IV-B)

def test_saddle_refinement_hand_case():
    g = load("h4_saddle.txt")
    a = grid(g["field"], np.float32).astype(np.float32)
    eps = float(g["eps"])
    assert (oracle.critical_points(a) == grid(g["labels"], int)).all()
    buf = oracle.compress(a, eps, rel=False, rbf_k=3, rbf_sigma=1.0)
    assert (bin_codes(a, buf) == grid(g["bins"], int)).all()
    h, w, hf = header_q(buf)
    out, d0, d1, stats = oracle.decompress(buf, a.shape, stages=True)
    assert (d0 == grid(g["bins"], int).astype(np.float32) * w).all()
    assert oracle.critical_points(d0)[2, 2] == R          # saddle lost by QZ^
    assert (d1 == d0).all()                               # no extrema stencil fires
    want = d0.copy()
    want[2, 2] = np.float32(w + np.float32(np.float32(0.1) * hf))
    assert (out == want).all()
    assert (oracle.critical_points(out) == grid(g["labels"], int)).all()
    assert stats[2] == 1


def _run_golden(name):
    g = load(name)
    a = field(g)
    p = tuple(int(v) for v in g["p"].split())
    buf = oracle.compress(a, float(g["eps"]), rel=False, rbf_k=int(g["rbf_k"]),
                          rbf_sigma=float(g["rbf_sigma"]))
    h, w, hf = header_q(buf)
    assert h["rbf_k"] == int(g["rbf_k"]) and np.float32(h["rbf_sigma"]) == np.float32(g["rbf_sigma"])
    out, d0, d1, stats = oracle.decompress(buf, a.shape, stages=True)
    return g, a, p, buf, w, hf, out, d0, d1, stats


@pytest.mark.parametrize("name", ["rs_shepard_2d_k5.txt", "rs_shepard_2d_k5_edge.txt"])
def test_saddle_shepard_value_hand_cases(name):
    """Section IV-B(3): the refined value is the normalised Gaussian kernel
    sum over N_r(p) minus p, restricted to the grid, with weights
    exp(-d^2 / 2 sigma^2) by squared distance; the fixtures give its offset
    from p in bin units, worked by hand.  The clamp does not bind there, so
    the output value of p is the kernel sum itself."""
    g, a, p, buf, w, hf, out, d0, d1, stats = _run_golden(name)
    labels = grid(g["labels"], int)
    assert (oracle.critical_points(a) == labels).all() and labels[p] == SAD
    assert (bin_codes(a, buf) == grid(g["bins"], int)).all()
    assert oracle.critical_points(d0)[p] == R                      # lost by QZ^
    r = int(g["rbf_k"]) // 2
    ball = np.sum((np.indices(a.shape) - np.array(p).reshape(-1, 1, 1)) ** 2, axis=0) <= r * r
    assert (d1[ball] == d0[ball]).all()                            # no stencil inside the ball
    # binary32 rounding: 12 products and sums of values ~0.13 (each within
    # 2^-24 relative) plus the final add, over w ~ 0.02: below 5e-6 of w
    step = (float(out[p]) - float(d0[p])) / float(w)
    assert abs(step - float(g["step_over_w"])) <= 5e-6, step
    changed = np.argwhere(out != d1)
    assert [tuple(c) for c in changed] == [p]
    assert (oracle.critical_points(out) == labels).all()
    assert stats[2] == 1


def test_saddle_clamp_3d_hand_case():
    """3D, k_size = 3: the kernel mean lies w/6 below p, the step limit
    0.1 h binds, and the move down makes p a saddle again (fixture)."""
    g, a, p, buf, w, hf, out, d0, d1, stats = _run_golden("rs_clamp_3d_k3.txt")
    lab = oracle.critical_points(a)
    assert (lab[2] == grid(g["labels_z2"], int)).all() and (lab[1] == R).all()
    assert (bin_codes(a, buf)[2] == grid(g["bins_z2"], int)).all()
    assert oracle.critical_points(d0)[p] == R
    assert out[p] == np.float32(d1[p] - np.float32(np.float32(0.1) * hf))
    assert [tuple(c) for c in np.argwhere(out != d1)] == [p]
    assert (oracle.critical_points(out) == lab).all()
    assert stats[2] == 1


def test_saddle_refused_when_a_neighbour_would_change_type():
    """End of Section IV-B: a correction that would create a critical point
    absent from the original map is suppressed (fixture): moving p down
    would make its x+ neighbour n a strict maximum."""
    g, a, p, buf, w, hf, out, d0, d1, stats = _run_golden("rs_reject_new_type_3d.txt")
    n = tuple(int(v) for v in g["n"].split())
    lab = oracle.critical_points(a)
    assert (lab[2] == grid(g["labels_z2"], int)).all() and lab[n] == R
    # the candidate of the hand derivation, checked by plain comparisons:
    v = np.float32(d1[p] - np.float32(np.float32(0.1) * hf))
    F = d1.copy()
    F[p] = v
    z, y, x = p
    assert F[z, y, x - 1] > v and F[z, y, x + 1] > v          # x pair higher
    assert F[z, y - 1, x] > v and F[z, y + 1, x] > v          # y pair higher
    assert F[z - 1, y, x] < v and F[z + 1, y, x] < v          # z pair lower: p a saddle
    nz, ny, nx = n
    nb = [F[nz, ny, nx - 1], F[nz, ny, nx + 1], F[nz, ny - 1, nx], F[nz, ny + 1, nx],
          F[nz - 1, ny, nx], F[nz + 1, ny, nx]]
    assert all(u < F[n] for u in nb)                          # n a new maximum
    assert d1[p] == d1[n]                                     # before the move: a tie
    # refused: p keeps its value and stays lost, nothing else moves
    assert (out == d1).all()
    assert stats[2] == 0
    lo = oracle.critical_points(out)
    assert lo[p] == R and lo[n] == R
    e = oracle.topo_errors(lab, lo)
    assert e[1].sum() == 0 and e[2].sum() == 0


@pytest.mark.parametrize("ndim", [2, 3])
def test_saddle_colouring_is_distance_two(ndim):
    """Within one colour round no two candidates may share a face neighbour, so
    every same-colour pair must be at Manhattan distance >= 3 (brute force over a
    patch larger than the colour period)."""
    rng = range(9)
    pts = list(itertools.product(rng, rng, range(9) if ndim == 3 else [0]))
    col = {p: oracle.colour(ndim, *p) for p in pts}
    assert {c[1] for c in col.values()} == {5 if ndim == 2 else 7}
    assert len({c[0] for c in col.values()}) == (5 if ndim == 2 else 7)
    for p in pts:
        for dx, dy, dz in itertools.product(range(-2, 3), repeat=3):
            if ndim == 2 and dz:
                continue
            dist = abs(dx) + abs(dy) + abs(dz)
            q = (p[0] + dx, p[1] + dy, p[2] + dz)
            if 0 < dist <= 2 and q in col:
                assert col[q][0] != col[p][0]


def test_exp_neg_against_libm():
    for t in np.linspace(0, 20, 401):
        e = oracle.exp_neg(float(t))
        assert abs(e - math.exp(-t)) <= 1e-12 * math.exp(-t)


def test_rbf_weights_in_header():
    a = synth.gaussian_bumps_2d(40, 40, count=5, seed=8).numpy()
    buf = oracle.compress(a, 1e-3, rel=True)
    h = oracle.header(buf)
    s = float(np.float32(h["rbf_sigma"]))
    assert 0.5 <= s <= 1.0 and h["rbf_k"] in (3, 5, 7)
    want = np.array([math.exp(-d2 / (2 * s * s)) for d2 in range(1, 10)], np.float32)
    assert np.allclose(h["g"], want, rtol=1e-6, atol=0)


def test_rbf_parameters_grow_with_smoothness():
    """Section IV-B(3): sigma in [0.5, 1] is larger for smooth data and the
    kernel size grows when the variation is low.  Along a family from smooth
    to rough (Gaussian random fields with flatter and flatter spectra, then
    white noise) neither may grow; a gentle ramp takes the largest kernel and
    white noise the smallest kernel and sigma.  (The thresholds themselves
    are the implementation's choice: the paper gives none.)"""
    ramp = (np.arange(1024, dtype=np.float64)[None, :] / 1024 +
            np.arange(64, dtype=np.float64)[:, None] / 640).astype(np.float32)
    fields = [ramp] + [synth.grf((128, 128), s, 7).numpy() for s in (-8, -4, -3, -2, -1)]
    fields.append(np.random.default_rng(5).random((128, 128)).astype(np.float32))
    ks, sig = [], []
    for a in fields:
        h = oracle.header(oracle.compress(a, 1e-3, rel=True))
        ks.append(h["rbf_k"])
        sig.append(float(np.float32(h["rbf_sigma"])))
    assert all(x >= y for x, y in zip(ks, ks[1:])), ks
    assert all(x >= y for x, y in zip(sig, sig[1:])), sig
    assert ks[0] == 7 and sig[0] > 0.95
    assert ks[-1] == 3 and sig[-1] == 0.5


def _ball_offsets(ndim, r):
    """N_r(p) minus p as (x, y, z) offsets, (z, y, x) ascending."""
    rz = r if ndim == 3 else 0
    return [(dx, dy, dz) for dz in range(-rz, rz + 1) for dy in range(-r, r + 1) for dx in range(-r, r + 1)
            if 0 < dx * dx + dy * dy + dz * dz <= r * r]


RBF_CASES = [(nd, r, s) for nd in (2, 3) for r in (1, 2, 3) for s in (0.5, 0.75, 1.0)]


@pytest.mark.parametrize("ndim,r,sigma", RBF_CASES)
def test_rbf_solve_equals_bordered_system(ndim, r, sigma):
    """Eqs. RBF-interp-final / RBF-eval with a constant term: the evaluation
    weights at p are the first m entries of M^-1 [phi_p; 1], M the bordered
    matrix [[Phi, 1], [1^T, 0]] -- solved here by LU on the whole bordered
    system, which the oracle never forms (it eliminates the constant by two
    Cholesky solves).  The condition number of Phi stays below 1e4 for every
    radius and width the compressor chooses, so 1e-10 relative is loose."""
    P = np.array(_ball_offsets(ndim, r), np.float64)
    m = len(P)
    D2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    Phi = np.exp(-D2 / (2 * sigma * sigma))
    M = np.ones((m + 1, m + 1))
    M[:m, :m] = Phi
    M[m, m] = 0.0
    rhs = np.append(np.exp(-(P ** 2).sum(-1) / (2 * sigma * sigma)), 1.0)
    want = np.linalg.solve(M, rhs)[:m]
    got = oracle.rbf_solve(ndim, r, sigma)
    assert got.shape == (m,) and m == {(2, 1): 4, (2, 2): 12, (2, 3): 28, (3, 1): 6, (3, 2): 32, (3, 3): 122}[(ndim, r)]
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max(), np.abs(got - want).max()
    assert abs(got.sum() - 1.0) <= 1e-13


@pytest.mark.parametrize("ndim,r,sigma", RBF_CASES)
def test_rbf_solve_interpolates_and_is_symmetric(ndim, r, sigma):
    """The interpolant passes through the data: evaluated at node j its
    weights are the unit vector e_j.  At p, the ball's symmetries (axis flips
    and, in the plane or cube, axis swaps) map nodes onto nodes, so nodes at
    the same distance from p get the same weight; hence linear functions are
    reproduced at p as well (sum alpha_i q_i = 0).  (Equal distance alone is
    not enough: (3, 0, 0) and (2, 2, 1) are not images of one another.)"""
    offs = _ball_offsets(ndim, r)
    for j in range(0, len(offs), max(1, len(offs) // 7)):
        w = oracle.rbf_solve(ndim, r, sigma, at=offs[j])
        e = np.zeros(len(offs))
        e[j] = 1.0
        assert np.abs(w - e).max() <= 1e-11, (j, np.abs(w - e).max())
    a = oracle.rbf_solve(ndim, r, sigma)
    orbit = [tuple(sorted(abs(c) for c in o)) for o in offs]
    for key in set(orbit):
        grp = a[[k == key for k in orbit]]
        assert np.ptp(grp) <= 1e-12, (key, grp)
    assert len(set(orbit)) < len(offs)
    assert np.abs((a[:, None] * np.array(offs, np.float64)).sum(0)).max() <= 1e-12


def test_rbf_solve_mode_only_moves_saddle_candidates():
    """The literal interpolation (header flag RBF_SOLVE) changes RS^ alone:
    against the default reading the decoded fields differ only at
    saddle-labelled points; FP = FT = 0 and the relaxed bound eps + h still
    hold, and the streams differ in the flag word alone."""
    for name, a in _fields_small():
        for eb in (1e-2, 1e-3):
            b0 = oracle.compress(a, eb, rel=True)
            b1 = oracle.compress(a, eb, rel=True, rbf_solve=True)
            assert oracle.header(b1)["flags"] == oracle.RBF_SOLVE
            diff = [i for i in range(len(b0)) if b0[i] != b1[i]]
            assert len(b0) == len(b1) and diff in ([], [40]), (name, diff)
            o0, o1 = oracle.decompress(b0, a.shape), oracle.decompress(b1, a.shape)
            la, l1 = oracle.critical_points(a), oracle.critical_points(o1)
            moved = o0.view(np.uint32) != o1.view(np.uint32)
            assert np.all(la[moved] == SAD), name
            err = oracle.topo_errors(la, l1)
            assert err[1].sum() == 0 and err[2].sum() == 0, (name, err)
            h = oracle.header(b1)
            dev = np.abs(a.astype(np.float64) - o1.astype(np.float64)).max()
            assert dev <= h["eps"] + float(np.float32(h["h_f"])) * (1 + 2 ** -20), name


def test_rbf_solve_needs_a_positive_width():
    """With the literal interpolation the decoder solves with the header's
    sigma: a width that is not a positive finite number marks the stream
    damaged."""
    import struct
    a = synth.gaussian_bumps_2d(20, 24, count=4, seed=1).numpy()
    buf = bytearray(oracle.compress(a, 1e-3, rel=True, rbf_solve=True))
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        buf[92:96] = struct.pack("<f", bad)
        with pytest.raises(oracle.OracleError) as ei:
            oracle.decompress(bytes(buf), a.shape)
        assert ei.value.status == oracle.CORRUPT


# ------------------------------------------------ format v2: tile-shaped blocks

def _sections(buf):
    h = oracle.header(buf)
    nb = h["nb"]
    width = np.frombuffer(buf[h["off_s2"]:h["off_s2"] + nb], np.uint8)
    first = np.frombuffer(buf[h["off_s4"]:h["off_s4"] + 4 * nb], "<i4")
    pay = np.frombuffer(buf[h["off_s5"]:h["off_s5"] + 4 * h["pay_words"]], "<u4")
    return h, width, first, pay


def test_tile_block_lorenzo_hand_case():
    """Format v2 (Section II-C's B + LZ on a tile-shaped block): one 8 x 4
    block of integer values with |a| <= 85 and absolute eps 0.5, so the bin
    width is just below 1 and every code equals its value.  The codes are
    q = 7 + 3x + 5y + 2xy.  Worked by hand:
    - Lorenzo residuals: 0 at the corner, 3 along row 0, 5 down column 0, and
      the mixed term 2 inside.  The widest is 5, so w = 3.
    - The element-order chain jumps by -16, -30 and -44 at the row starts, so
      Lorenzo is coded: width byte 0x83, first value 7.
    - Payload: the sign plane 0, then magnitude planes 0x010101FE (bit 0: the
      3s and 5s), 0xFEFEFEFE (bit 1: the 3s and 2s), 0x01010100 (bit 2: the 5s)."""
    y, x = np.mgrid[0:4, 0:8]
    a = (7 + 3 * x + 5 * y + 2 * x * y).astype(np.float32)
    buf = oracle.compress(a, 0.5, rel=False, no_topo=True, tile_blocks=True)
    h, width, first, pay = _sections(buf)
    assert h["version"] == 2 and h["nb"] == 1
    assert width.tolist() == [0x83] and first.tolist() == [7]
    assert pay.tolist() == [0, 0x010101FE, 0xFEFEFEFE, 0x01010100]
    out = oracle.decompress(buf, a.shape)
    assert np.abs(out.astype(np.float64) - a).max() <= 0.5


def test_tile_block_chain_hand_case():
    """Rows 0 1 0 1 ... repeated in every row: the chain's residuals are
    +1 (odd e) and -1 (even e > 0), width 1; Lorenzo's are +-1 along row 0
    and 0 elsewhere, also width 1.  On a tie the chain is coded: width byte
    0x01, sign plane 0x55555554 (the even e > 0), magnitude plane 0xFFFFFFFE."""
    a = np.tile(np.array([0, 1] * 4, np.float32), (4, 1))
    buf = oracle.compress(a, 0.5, rel=False, no_topo=True, tile_blocks=True)
    h, width, first, pay = _sections(buf)
    assert width.tolist() == [0x01] and first.tolist() == [0]
    assert pay.tolist() == [0x55555554, 0xFFFFFFFE]


def _tile_cases():
    rng = np.random.default_rng(11)
    yield "bumps", synth.gaussian_bumps_2d(64, 80, count=20, seed=5).numpy()
    yield "climate", synth.climate_2d(61, 97, seed=2).numpy()
    yield "turb", synth.turbulence_3d(20, seed=3).numpy()
    yield "ragged3", synth.grf((7, 9, 13), -11 / 3, 4).numpy()
    yield "adv2", synth.adversarial_small(1, (33, 17)).numpy()
    yield "adv3", synth.adversarial_small(2, (9, 8, 7)).numpy()
    for shape in [(1, 1), (1, 37), (37, 1), (3, 3), (1, 1, 40), (5, 1, 7), (40, 1, 1), (2, 3, 5)]:
        yield f"rand{shape}", rng.standard_normal(shape).astype(np.float32)
    yield "checker", ((1.0 + rng.random((10, 12))) * np.where(np.indices((10, 12)).sum(0) % 2, 1.0, -1.0)).astype(np.float32)


@pytest.mark.parametrize("opts", [dict(rel=True, eb=1e-2), dict(rel=True, eb=1e-4), dict(rel=False, eb=0.05),
                                  dict(rel=True, eb=1e-3, no_topo=True)])
def test_tile_format_decodes_to_the_format_v1_field(opts):
    """Format v2 changes only how the codes are coded: the decoded field, the
    labels and the rank stream equal format v1's bit for bit, on 2D and 3D
    fields, ragged and one-point-thin grids (where most of a block lies
    outside the grid and takes clamped codes), and for both bound modes."""
    for name, a in _tile_cases():
        b1 = oracle.compress(a, **opts)
        b2 = oracle.compress(a, tile_blocks=True, **opts)
        h1, h2 = oracle.header(b1), oracle.header(b2)
        assert h1["version"] == 1 and h2["version"] == 2, name
        assert h2["nb"] == oracle.tile_blocks(a.shape), name
        assert h1["sum_abs"] == h2["sum_abs"] and h1["rbf_k"] == h2["rbf_k"], name
        if not opts.get("no_topo"):
            n = a.size
            lab1 = b1[h1["off_s6"]:h1["off_s6"] + 4 * ((n + 15) // 16)]
            lab2 = b2[h2["off_s6"]:h2["off_s6"] + 4 * ((n + 15) // 16)]
            assert lab1 == lab2, name
            assert b1[h1["off_s7"]:h1["total"]] == b2[h2["off_s7"]:h2["total"]], name
        o1, o2 = oracle.decompress(b1, a.shape), oracle.decompress(b2, a.shape)
        assert np.array_equal(o1.view(np.uint32), o2.view(np.uint32)), name


def test_tile_blocks_count_and_bound():
    """Blocks of format v2: ceil(nx/8) ceil(ny/4) in 2D, ceil(nx/4) ceil(ny/4)
    ceil(nz/2) in 3D; the compression bound covers either format."""
    assert oracle.tile_blocks((4, 8)) == 1 and oracle.tile_blocks((5, 9)) == 4
    assert oracle.tile_blocks((37, 1)) == 10 and oracle.tile_blocks((1, 37)) == 5
    assert oracle.tile_blocks((2, 4, 4)) == 1 and oracle.tile_blocks((3, 5, 5)) == 8
    assert oracle.tile_blocks((40, 1, 1)) == 20
    rng = np.random.default_rng(3)
    for shape in [(1, 1000), (1000, 1), (1, 1, 300), (300, 1, 1), (17, 23, 5)]:
        a = rng.standard_normal(shape).astype(np.float32)
        assert len(oracle.compress(a, 1e-5, tile_blocks=True)) <= oracle.compress_bound(shape)


def test_tile_blocks_code_smooth_fields_smaller():
    """On the smooth synthetic fields the tile-shaped blocks code fewer
    payload words than runs of 32 consecutive points (same decoded field)."""
    for name, a in (("turb", synth.turbulence_3d(32, seed=3).numpy()),
                    ("bumps", synth.gaussian_bumps_2d(96, 128, count=20, seed=5).numpy())):
        for eb in (1e-3, 1e-4):
            p1 = oracle.header(oracle.compress(a, eb, no_topo=True))["pay_words"]
            p2 = oracle.header(oracle.compress(a, eb, no_topo=True, tile_blocks=True))["pay_words"]
            assert p2 < p1, (name, eb, p1, p2)


def test_tile_stream_damage_rejected():
    """A format-v2 width byte with the predictor bit but no planes, and a
    format-v1 stream relabelled as version 2 (its block count no longer
    matches the grid's tiles), mark the stream damaged."""
    import struct
    a = synth.gaussian_bumps_2d(20, 24, count=4, seed=1).numpy()
    buf = bytearray(oracle.compress(a, 1e-3, tile_blocks=True))
    h = oracle.header(bytes(buf))
    w = np.frombuffer(bytes(buf[h["off_s2"]:h["off_s2"] + h["nb"]]), np.uint8)
    j = int(np.nonzero(w == 0)[0][0]) if (w == 0).any() else None
    if j is not None:
        bad = bytearray(buf)
        bad[h["off_s2"] + j] = 0x80
        with pytest.raises(oracle.OracleError):
            oracle.decompress(bytes(bad), a.shape)
    b = synth.gaussian_bumps_2d(21, 24, count=4, seed=1).numpy()   # 16 runs of 32, 18 tiles
    v1 = bytearray(oracle.compress(b, 1e-3))
    v1[4:8] = struct.pack("<I", 2)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.decompress(bytes(v1), b.shape)
    assert ei.value.status == oracle.CORRUPT


def _fields_small():
    yield "bumps", synth.gaussian_bumps_2d(64, 80, count=20, seed=5).numpy()
    yield "climate", synth.climate_2d(60, 96, seed=2).numpy()
    yield "turb", synth.turbulence_3d(20, seed=3).numpy()
    yield "adv2", synth.adversarial_small(1, (33, 17)).numpy()
    yield "adv3", synth.adversarial_small(2, (9, 8, 7)).numpy()


@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4])
def test_invariants_no_fp_no_ft_bound(eb):
    """Section III-B / Table II: TopoSZp output has zero FP and zero FT; lost
    extrema are all restored unless the bound forbids it (counted); the
    relaxed bound |a - a'| <= eps + h < 2 eps holds (Table I, eps_topo)."""
    for name, a in _fields_small():
        buf = oracle.compress(a, eb, rel=True)
        h = oracle.header(buf)
        out, d0, d1, stats = oracle.decompress(buf, a.shape, stages=True)
        la, lo, l0 = (oracle.critical_points(x) for x in (a, out, d0))
        err = oracle.topo_errors(la, lo)
        assert err[1].sum() == 0 and err[2].sum() == 0, (name, err)
        assert err[0][MIN] + err[0][MAX] == stats[1], (name, err, stats)
        e0 = oracle.topo_errors(la, l0)
        assert e0[1].sum() == 0 and e0[2].sum() == 0          # SZp alone: FN only
        assert err[0].sum() <= e0[0].sum()
        dev = np.abs(a.astype(np.float64) - out.astype(np.float64)).max()
        assert dev <= h["eps"] + float(np.float32(h["h_f"])) * (1 + 2 ** -20)
        assert dev <= 2 * h["eps"]
        assert np.abs(a.astype(np.float64) - d0).max() <= h["eps"]


def test_szp_only_fn_has_same_bin_neighbour():
    """Section III-B: a critical point can only be lost when a neighbour shares
    its bin; with the topology layers switched off, FP = FT = 0."""
    a = synth.climate_2d(50, 80, seed=6).numpy()
    buf = oracle.compress(a, 1e-2, rel=True, no_topo=True)
    out = oracle.decompress(buf, a.shape)
    la, lo = oracle.critical_points(a), oracle.critical_points(out)
    q = bin_codes(a, buf)
    e = oracle.topo_errors(la, lo)
    assert e[1].sum() == 0 and e[2].sum() == 0 and e[0].sum() > 0
    ny, nx = a.shape
    for y, x in zip(*np.nonzero((la != R) & (lo == R))):
        nb = [(y + dy, x + dx) for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1))
              if 0 <= y + dy < ny and 0 <= x + dx < nx]
        assert any(q[j] == q[y, x] for j in nb)


def test_topo_errors_brute_force():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 4, 500).astype(np.uint8)
    b = rng.integers(0, 4, 500).astype(np.uint8)
    got = oracle.topo_errors(a, b)
    want = np.zeros((3, 4), np.uint64)
    for x, y in zip(a, b):
        if x != y:
            if y == R:
                want[0, x] += 1
            elif x == R:
                want[1, y] += 1
            else:
                want[2, x] += 1
    assert (got == want).all()


def test_corrupt_stream_rejected():
    a = synth.gaussian_bumps_2d(20, 24, count=4, seed=1).numpy()
    buf = bytearray(oracle.compress(a, 1e-3, rel=True))
    for bad in (bytes(buf[:100]), bytes(b"XXXX" + buf[4:])):
        with pytest.raises(oracle.OracleError):
            oracle.decompress(bad, a.shape)
    with pytest.raises(oracle.OracleError):
        oracle.decompress(bytes(buf), (a.shape[0] + 1, a.shape[1]))


@pytest.mark.parametrize("offset,value", [
    (40, 4),                  # flags: only NO_TOPO and RBF_SOLVE are defined
    (96, 0), (96, 17),        # RS^ sweeps outside 1..16
    (64, 0x7F800000),         # bin width w = +inf
    (72, 0xBF800000),         # half-width h < 0
    (120, 10 ** 6),           # more minima than half the points
    (160, 0),                 # section (2) offset off the layout
    (192, 7),                 # section (7) offset off the layout
])
def test_header_outside_what_compression_writes_is_corrupt(offset, value):
    """A header field outside the range compression gives it marks a damaged
    stream (stream layout, Section IV-A): the decoder refuses it rather than
    running e.g. 2^31 sweeps."""
    import struct
    a = synth.gaussian_bumps_2d(20, 24, count=4, seed=1).numpy()
    buf = bytearray(oracle.compress(a, 1e-3, rel=True))
    width = 8 if offset in (120, 160, 192) else 4
    buf[offset:offset + width] = struct.pack("<Q" if width == 8 else "<I", value)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.decompress(bytes(buf), a.shape)
    assert ei.value.status == oracle.CORRUPT
