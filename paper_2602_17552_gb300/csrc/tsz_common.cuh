// tsz_common.cuh -- device-side building blocks shared by the TopoSZp kernels.
//
// Everything here is compiled with --fmad=false, -ftz=false, -prec-div=true:
// each float expression below is one IEEE-754 binary32 (or binary64) operation
// rounded to nearest, so results are reproducible bit for bit.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tsz {

constexpr uint32_t L = 32;               // block length of the B stage (Section II-C)
constexpr uint32_t HDR = 256;            // stream header bytes
constexpr uint32_t MAGIC = 0x505A5354u;  // "TSZP"
constexpr uint32_t VERSION = 1;         // blocks of L consecutive points
constexpr uint32_t VERSION_TILES = 2;   // format v2: tile-shaped blocks (see tile_shape)
constexpr uint32_t FLAG_NO_TOPO = 1;
constexpr uint32_t FLAG_RBF_SOLVE = 2;   // RS^ by the literal interpolant's weights, unclamped
// Format v2 in the control block's flags (the stream itself says version 2;
// the header's flag word keeps only the two bits above).
constexpr uint32_t FLAG_TILE_BLOCKS = 4;
constexpr int RBF_MAX_NODES = 122;       // |N_r(p) \ {p}| for r = 3 in 3D

// labels of Section IV-A(1): r = 00, m = 01, s = 10, M = 11
constexpr int LAB_R = 0, LAB_MIN = 1, LAB_SAD = 2, LAB_MAX = 3;

// status codes (same values as toposzp_status)
constexpr int ST_OK = 0, ST_INVALID = 1, ST_NONFINITE = 2, ST_EB_SMALL = 3, ST_BUF_SMALL = 4,
              ST_CORRUPT = 5, ST_TIMEOUT = 6;

// Codec tile: one CTA of 8 warps, each warp owns 8 consecutive blocks of 32.
constexpr int TILE_WARPS = 8;
constexpr int BPW = 8;
constexpr int TILE_BLOCKS = TILE_WARPS * BPW;   // 64 blocks = 2048 points
constexpr int ENC_TILE_BLOCKS = 256;            // the field encoder's tile: 8192 points
constexpr uint32_t FULL = 0xFFFFFFFFu;

// Bounded waits: a look-back spin gives up after this many polls (each poll
// sleeps up to 256 ns), sets ST_TIMEOUT and lets the kernel finish.
constexpr uint32_t SPIN_LIMIT = 1u << 22;

__host__ __device__ constexpr inline uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
template <class T>
__host__ __device__ inline T hmin(T a, T b) { return a < b ? a : b; }
template <class T>
__host__ __device__ inline T hmax(T a, T b) { return a < b ? b : a; }
__host__ __device__ inline uint64_t align16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

// Division by a run-time invariant d by multiply-high and shifts (the
// round-up method of Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994): exact for every 32-bit dividend.
struct FastDiv {
    uint32_t d, m, s1, s2;
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) l++;                 // l = ceil(log2 d)
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 0 ? l - 1 : 0;
    return f;
}

__host__ __device__ inline uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.m, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct Geo {
    int ndim;
    uint32_t nx, ny, nz;   // nz = 1 in 2D
    uint32_t n;            // nx * ny * nz < 2^31
    uint32_t nxy;
    uint32_t nb;           // blocks of L
    FastDiv fx, fy;        // division by nx and by ny
};

// Format v2 blocks: L = 32 points shaped 8 x 4 in 2D and 4 x 4 x 2 in 3D (x
// fastest), in raster order over the block grid; element e of a block sits
// at (e mod BX, (e / BX) mod BY, e / (BX BY)) inside it.
template <int ND>
struct TileShape {
    static constexpr uint32_t BX = ND == 3 ? 4u : 8u, BY = 4u, BZ = ND == 3 ? 2u : 1u;
};
__host__ __device__ inline uint64_t tile_blocks(int ndim, uint64_t nx, uint64_t ny, uint64_t nz) {
    const uint64_t bx = ndim == 3 ? 4 : 8, by = 4, bz = ndim == 3 ? 2 : 1;
    return ((nx + bx - 1) / bx) * ((ny + by - 1) / by) * ((nz + bz - 1) / bz);
}

__host__ __device__ inline void geo_divs(Geo& g) {
    g.fx = make_fastdiv(g.nx);
    g.fy = make_fastdiv(g.ny);
}

// Stream layout of Section IV-A as placed in this format: header, (1) const
// bitmap, (2) widths, (4) first values, (6) labels, (3)+(5) planes, (7) ranks.
struct Layout {
    uint64_t s1, s2, s4, s6, s5, s5_end, s7, r1, r2, r4, r5, end;
};

__host__ __device__ inline void make_layout(uint64_t n, uint64_t nb, bool topo, uint64_t pay_words,
                                            uint64_t k, uint64_t rank_words, Layout& lo) {
    lo.s1 = HDR;
    lo.s2 = align16(lo.s1 + 4 * cdiv(nb, 32));
    lo.s4 = align16(lo.s2 + nb);
    lo.s6 = align16(lo.s4 + 4 * nb);
    lo.s5 = align16(lo.s6 + (topo ? 4 * cdiv(n, 16) : 0));
    lo.s5_end = lo.s5 + 4 * pay_words;
    if (topo) {
        uint64_t nbd = cdiv(k, L);
        lo.s7 = align16(lo.s5_end);
        lo.r1 = lo.s7;
        lo.r2 = align16(lo.r1 + 4 * cdiv(nbd, 32));
        lo.r4 = align16(lo.r2 + nbd);
        lo.r5 = align16(lo.r4 + 4 * nbd);
        lo.end = lo.r5 + 4 * rank_words;
    } else {
        lo.s7 = lo.r1 = lo.r2 = lo.r4 = lo.r5 = lo.end = lo.s5_end;
    }
}

// Device control block, first bytes of every workspace; zeroed by the host
// wrapper before the first kernel of a call.
struct Ctrl {
    // range pass
    unsigned int min_inv, max_key, nonfinite, sort_passes;
    unsigned int rank_bitmap, bm_words, bm_off, bin_n;   // dense ranks from key bitmaps (1) or the sort (0)
    // quantiser (Section II-C) and geometry, filled by the parameter kernel or
    // by the header parser
    int const_field, rel, rbf_k, rs_sweeps;
    float w_f, r_f, h_f, rbf_sigma;
    float vmin, vmax;
    uint32_t flags, pad1;
    double eps, eb;
    Geo g;
    // tile allocators of the persistent codec kernels
    // extrema lists (compress) and counts
    unsigned int cnt_max, cnt_min;
    int bin_q0;   // first QZ bin of the per-bin rank table (bin_n bins, 0: no table)
    unsigned int pad3;
    unsigned long long sum_abs;
    unsigned long long pay_words, k_total, rank_words, k_sad;
    unsigned long long counts[4];
    // decode-side bookkeeping
    unsigned long long stat_restored, stat_skipped, stat_saddle;
    unsigned int sad_cnt[8];
    unsigned int front[4];    // per-stage frontiers of the fused decoder
    unsigned int tile_fused, test_hold, pad5[2];   // test_hold: tile + 1 never published (0: none)
    unsigned int sad_col[8], sad_fill[8];   // lost saddles per colour (RS^ rounds)
    // per-slice sums of the tile counts (field tiles, rank-stream tiles), added
    // by the kernels that count, read by the slice-parallel scans
    unsigned long long sl_tile[32][2], sl_rank[32][2];
    unsigned int sad_next[8];               // work counters of the rounds' evaluation
    Layout lo;
    float g_rbf[9];
    float rbf_alpha[RBF_MAX_NODES];   // FLAG_RBF_SOLVE: the interpolant's weights at p, table order
    uint32_t nb_fmt;                  // blocks of the stream (g.nb in format v1, the tiles in v2)
};

// ------------------------------------------------------------------ helpers

// Programmatic dependent launch: the kernels of the library are launched with
// programmatic stream serialisation (launch_pdl) and start with
// griddep_enter(): it lets the next kernel's CTAs be scheduled once all of
// its own CTAs have started, then waits until every earlier kernel of the
// stream has completed and its writes are visible.  A launch thus overlaps
// the previous kernel's tail instead of following it; no memory access moves
// before the wait.  (Without the launch attribute the wait returns at once.)
__device__ __forceinline__ void griddep_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}


__device__ __forceinline__ void set_status(int* st, int code) {
    if (code) atomicCAS(st, 0, code);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Order-preserving map of binary32 onto uint32 (-0 folded onto +0).
__device__ __forceinline__ uint32_t ord_key(float v) {
    uint32_t b = __float_as_uint(v);
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(b);
}

// QZ: round-half-up of a / w as floor(fl(fl(a * r) + 0.5)) (Section II-C).
__device__ __forceinline__ int32_t quantize(float a, float r) {
    float x = __fmul_rn(a, r);
    float y = __fadd_rn(x, 0.5f);
    return (int32_t)floorf(y);
}
// QZ^: bin centre q * w.
__device__ __forceinline__ float dequantize(int32_t q, float w) {
    return __fmul_rn(__int2float_rn(q), w);
}

// gather the even bit positions of x into the low 16 bits (inverse of spread16)
__device__ __forceinline__ uint32_t compact16(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// Exclusive scan of pairs (a_i, b_i), i < cnt, by one CTA of 1024 threads:
// chunks of 4096 entries, four consecutive entries per thread, a shuffle scan
// of the threads' sums per warp, one shared step per chunk, running 64-bit
// carries.  load(i) -> uint2; store(i, pa, pb).  Returns the totals.  Shared
// scratch: s_w[33] pairs.
template <class Load, class Store>
__device__ void cta_scan_pairs(uint32_t cnt, Load load, Store store, unsigned long long (*s_w)[2],
                               unsigned long long& tot_a, unsigned long long& tot_b) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t PER = 4, CHUNK = 1024 * PER;
    unsigned long long ca = 0, cb = 0;
    for (uint32_t base = 0; base < cnt; base += CHUNK) {
        const uint32_t i0 = base + threadIdx.x * PER;
        uint2 v[PER];
        unsigned long long sa = 0, sb = 0;
#pragma unroll
        for (uint32_t j = 0; j < PER; j++) {
            v[j] = i0 + j < cnt ? load(i0 + j) : make_uint2(0u, 0u);
            sa += v[j].x;
            sb += v[j].y;
        }
        unsigned long long ia = sa, ib = sb;
#pragma unroll
        for (int of = 1; of < 32; of <<= 1) {
            const unsigned long long ta = __shfl_up_sync(0xFFFFFFFFu, ia, of), tb = __shfl_up_sync(0xFFFFFFFFu, ib, of);
            if (lane >= (uint32_t)of) { ia += ta; ib += tb; }
        }
        if (lane == 31) { s_w[warp][0] = ia; s_w[warp][1] = ib; }
        __syncthreads();
        if (warp == 0) {   // exclusive prefixes of the 32 warp totals, and the chunk total
            const unsigned long long xa = s_w[lane][0], xb = s_w[lane][1];
            unsigned long long ra = xa, rb = xb;
#pragma unroll
            for (int of = 1; of < 32; of <<= 1) {
                const unsigned long long ta = __shfl_up_sync(0xFFFFFFFFu, ra, of), tb = __shfl_up_sync(0xFFFFFFFFu, rb, of);
                if (lane >= (uint32_t)of) { ra += ta; rb += tb; }
            }
            s_w[lane][0] = ra - xa;
            s_w[lane][1] = rb - xb;
            if (lane == 31) { s_w[32][0] = ra; s_w[32][1] = rb; }
        }
        __syncthreads();
        unsigned long long pa = ca + s_w[warp][0] + ia - sa, pb = cb + s_w[warp][1] + ib - sb;
#pragma unroll
        for (uint32_t j = 0; j < PER; j++) {
            if (i0 + j < cnt) store(i0 + j, pa, pb);
            pa += v[j].x;
            pb += v[j].y;
        }
        ca += s_w[32][0];
        cb += s_w[32][1];
        __syncthreads();
    }
    tot_a = ca;
    tot_b = cb;
}

// Slice-parallel form: SCAN_SLICES CTAs, CTA j scans entries [j * len, (j +
// 1) * len) of [0, cnt), len = slice_len(cnt), offset by the sums of the
// slices before it; the sums (sl[j] = {sum a, sum b} of slice j) were added
// up by the kernel that wrote the entries.  No CTA waits on another.  Returns
// the totals over all slices.
constexpr uint32_t SCAN_SLICES = 32;
__host__ __device__ inline uint32_t slice_len(uint32_t cnt) {
    const uint32_t l = (cnt + SCAN_SLICES - 1) / SCAN_SLICES;
    return l ? l : 1u;
}
template <class Load, class Store>
__device__ void slice_scan_pairs(uint32_t cnt, const unsigned long long (*sl)[2], Load load, Store store,
                                 unsigned long long (*s_w)[2], unsigned long long& tot_a,
                                 unsigned long long& tot_b) {
    __shared__ unsigned long long s_off[4];
    const uint32_t j = blockIdx.x;
    if (threadIdx.x < 32) {
        const unsigned long long xa = sl[threadIdx.x][0], xb = sl[threadIdx.x][1];
        unsigned long long oa = 0, ob = 0, ta = 0, tb = 0;
        for (uint32_t i = 0; i < SCAN_SLICES; i++) {
            const unsigned long long ya = __shfl_sync(FULL, xa, i), yb = __shfl_sync(FULL, xb, i);
            if (i < j) { oa += ya; ob += yb; }
            ta += ya;
            tb += yb;
        }
        if (threadIdx.x == 0) {
            s_off[0] = oa;
            s_off[1] = ob;
            s_off[2] = ta;
            s_off[3] = tb;
        }
    }
    __syncthreads();
    const unsigned long long oa = s_off[0], ob = s_off[1];
    tot_a = s_off[2];
    tot_b = s_off[3];
    const uint32_t len = slice_len(cnt);
    const uint32_t lo = j * len < cnt ? j * len : cnt;
    const uint32_t hi = cnt - lo < len ? cnt : lo + len;
    unsigned long long sa, sb;
    cta_scan_pairs(
        hi - lo, [&](uint32_t i) { return load(lo + i); },
        [&](uint32_t i, unsigned long long pa, unsigned long long pb) { store(lo + i, oa + pa, ob + pb); }, s_w, sa,
        sb);
    __syncthreads();   // s_off and s_w are free again
}

// ---------------------------------------------------- bit-plane transposes
//
// A block's fixed-length code (Section II-C, BE) stores w bit planes: plane r
// holds bit r of value e at bit e.  Values and planes are the rows and
// columns of a bit matrix, so one turns into the other by a transpose done in
// registers with the recursive block swap (H. S. Warren, "Hacker's Delight",
// section 7-3): log2(k) rounds of masked shift-and-xor exchanges, instead of
// one instruction per bit.  Narrow blocks use four 8x8 (or two 16x16)
// matrices side by side in the byte (half-word) lanes of the same words: the
// masks keep the lanes apart.  W, the width that picks the variant, is the
// same for the whole warp (the branch is uniform); it bounds every block's
// own width w.

template <int S>
__device__ __forceinline__ void bt_swap(uint32_t& a, uint32_t& b, uint32_t m) {
    const uint32_t t = ((a >> S) ^ b) & m;
    b ^= t;
    a ^= t << S;
}

// four independent 8x8 transposes, one per byte lane of x[0..7]
__device__ __forceinline__ void bt8x4(uint32_t (&x)[8]) {
#pragma unroll
    for (int i = 0; i < 4; i++) bt_swap<4>(x[i], x[i + 4], 0x0F0F0F0Fu);
#pragma unroll
    for (int i = 0; i < 8; i++)
        if ((i & 2) == 0) bt_swap<2>(x[i], x[i + 2], 0x33333333u);
#pragma unroll
    for (int i = 0; i < 8; i += 2) bt_swap<1>(x[i], x[i + 1], 0x55555555u);
}

// two independent 16x16 transposes, one per half-word lane of x[0..15]
__device__ __forceinline__ void bt16x2(uint32_t (&x)[16]) {
#pragma unroll
    for (int i = 0; i < 8; i++) bt_swap<8>(x[i], x[i + 8], 0x00FF00FFu);
#pragma unroll
    for (int i = 0; i < 16; i++)
        if ((i & 4) == 0) bt_swap<4>(x[i], x[i + 4], 0x0F0F0F0Fu);
#pragma unroll
    for (int i = 0; i < 16; i++)
        if ((i & 2) == 0) bt_swap<2>(x[i], x[i + 2], 0x33333333u);
#pragma unroll
    for (int i = 0; i < 16; i += 2) bt_swap<1>(x[i], x[i + 1], 0x55555555u);
}

// one 32x32 transpose of x[0..31]
__device__ __forceinline__ void bt32(uint32_t (&x)[32]) {
#pragma unroll
    for (int i = 0; i < 16; i++) bt_swap<16>(x[i], x[i + 16], 0x0000FFFFu);
#pragma unroll
    for (int i = 0; i < 32; i++)
        if ((i & 8) == 0) bt_swap<8>(x[i], x[i + 8], 0x00FF00FFu);
#pragma unroll
    for (int i = 0; i < 32; i++)
        if ((i & 4) == 0) bt_swap<4>(x[i], x[i + 4], 0x0F0F0F0Fu);
#pragma unroll
    for (int i = 0; i < 32; i++)
        if ((i & 2) == 0) bt_swap<2>(x[i], x[i + 2], 0x33333333u);
#pragma unroll
    for (int i = 0; i < 32; i += 2) bt_swap<1>(x[i], x[i + 1], 0x55555555u);
}

// The 32 magnitudes of a block from its w planes (plane(r), r < w); W >= w.
template <class Plane>
__device__ __forceinline__ void planes_to_values(uint32_t W, uint32_t w, const Plane& plane, uint32_t (&v)[32]) {
    if (W <= 8) {
        uint32_t x[8];
#pragma unroll
        for (int r = 0; r < 8; r++) x[r] = (uint32_t)r < w ? plane(r) : 0u;
        bt8x4(x);
#pragma unroll
        for (int e = 0; e < 32; e++) v[e] = (x[e & 7] >> (8 * (e >> 3))) & 0xFFu;
    } else if (W <= 16) {
        uint32_t x[16];
#pragma unroll
        for (int r = 0; r < 16; r++) x[r] = (uint32_t)r < w ? plane(r) : 0u;
        bt16x2(x);
#pragma unroll
        for (int e = 0; e < 32; e++) v[e] = (x[e & 15] >> (16 * (e >> 4))) & 0xFFFFu;
    } else {
#pragma unroll
        for (int r = 0; r < 32; r++) v[r] = (uint32_t)r < w ? plane(r) : 0u;
        bt32(v);
    }
}

// The w planes of a block from its 32 magnitudes (each below 2^W), handed to
// put(r, plane) for r < w.
template <class Put>
__device__ __forceinline__ void values_to_planes(uint32_t W, uint32_t w, const uint32_t (&m)[32], const Put& put) {
    if (W <= 8) {
        uint32_t x[8];
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = m[i] | m[8 + i] << 8 | m[16 + i] << 16 | m[24 + i] << 24;
        bt8x4(x);
#pragma unroll
        for (int r = 0; r < 8; r++)
            if ((uint32_t)r < w) put(r, x[r]);
    } else if (W <= 16) {
        uint32_t x[16];
#pragma unroll
        for (int i = 0; i < 16; i++) x[i] = m[i] | m[16 + i] << 16;
        bt16x2(x);
#pragma unroll
        for (int r = 0; r < 16; r++)
            if ((uint32_t)r < w) put(r, x[r]);
    } else {
        uint32_t x[32];
#pragma unroll
        for (int i = 0; i < 32; i++) x[i] = m[i];
        bt32(x);
#pragma unroll
        for (int r = 0; r < 32; r++)
            if ((uint32_t)r < w) put(r, x[r]);
    }
}

// spread the low 16 bits of x to the even bit positions
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__device__ __forceinline__ int label_at(const uint32_t* labels, uint32_t i) {
    return (int)((labels[i >> 4] >> ((i & 15u) * 2u)) & 3u);
}

// CD of Section IV-A(1) at point i with coordinates (x, y, z): strict
// comparisons with the face neighbours inside the grid.  m: all higher; M: all
// lower; s: both neighbours on every axis, each pair entirely higher (H) or
// entirely lower (L), at least one H and one L pair (the 2D rule of the paper
// and its 3D extension).  `val(j)` returns the field value at index j.
template <class Val>
__device__ __forceinline__ int classify(const Val& val, const Geo& g, uint32_t i, uint32_t x,
                                        uint32_t y, uint32_t z, float v) {
    int nn = 0, nhi = 0, nlo = 0, ph = 0, pl = 0, px = 0;
    bool interior = true;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        if (ax == 2 && g.ndim != 3) break;
        uint32_t c = ax == 0 ? x : (ax == 1 ? y : z);
        uint32_t d = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
        uint32_t s = ax == 0 ? 1u : (ax == 1 ? g.nx : g.nxy);
        bool lo = c > 0, hi = c + 1 < d;
        int hc = 0, lc = 0;
        if (lo) {
            float u = val(i - s);
            nn++;
            if (u > v) { nhi++; hc++; } else if (u < v) { nlo++; lc++; }
        }
        if (hi) {
            float u = val(i + s);
            nn++;
            if (u > v) { nhi++; hc++; } else if (u < v) { nlo++; lc++; }
        }
        if (lo && hi) {
            if (hc == 2) ph++;
            else if (lc == 2) pl++;
            else px++;
        } else {
            interior = false;
        }
    }
    if (nn == 0) return LAB_R;
    if (nhi == nn) return LAB_MIN;
    if (nlo == nn) return LAB_MAX;
    if (interior && px == 0 && ph > 0 && pl > 0) return LAB_SAD;
    return LAB_R;
}

struct GlobalVal {
    const float* F;
    __device__ __forceinline__ float operator()(uint32_t j) const { return F[j]; }
};

__device__ __forceinline__ void coords(const Geo& g, uint32_t i, uint32_t& x, uint32_t& y,
                                       uint32_t& z) {
    const uint32_t t = fdiv(i, g.fx);
    x = i - t * g.nx;
    z = fdiv(t, g.fy);
    y = t - z * g.ny;
}

// classify() for a point known to have both neighbours on every axis: the same
// rule as a straight-line sequence of comparisons.
template <class Val>
__device__ __forceinline__ int classify_interior(const Val& val, const Geo& g, uint32_t i, float v) {
    const float xm = val(i - 1), xp = val(i + 1), ym = val(i - g.nx), yp = val(i + g.nx);
    const bool three = g.ndim == 3;
    const float zm = three ? val(i - g.nxy) : xm, zp = three ? val(i + g.nxy) : xp;
    const bool Hx = xm > v && xp > v, Lx = xm < v && xp < v;
    const bool Hy = ym > v && yp > v, Ly = ym < v && yp < v;
    const bool Hz = !three || (zm > v && zp > v), Lz = !three || (zm < v && zp < v);
    const bool m = Hx && Hy && Hz, M = Lx && Ly && Lz;
    const bool s = (Hx || Lx) && (Hy || Ly) && (Hz || Lz) && !m && !M;
    return (int)((uint32_t)(m | M) | ((uint32_t)(s | M) << 1));
}

__device__ __forceinline__ bool is_interior(const Geo& g, uint32_t x, uint32_t y, uint32_t z) {
    return x > 0 && x + 1 < g.nx && y > 0 && y + 1 < g.ny && (g.ndim == 2 || (z > 0 && z + 1 < g.nz));
}

template <class Val>
__device__ __forceinline__ int classify_any(const Val& val, const Geo& g, uint32_t i, uint32_t x, uint32_t y,
                                            uint32_t z, float v) {
    return is_interior(g, x, y, z) ? classify_interior(val, g, i, v) : classify(val, g, i, x, y, z, v);
}


// exp(-t), t >= 0, by scaling and squaring with a 12-term Taylor polynomial:
// only binary64 + * /, so host and device give identical bits.
__host__ __device__ inline double exp_neg(double t) {
#ifdef __CUDA_ARCH__
    double y = __ddiv_rn(-t, 1024.0);
    double e = 1.0;
    for (int j = 12; j >= 1; j--) e = __dadd_rn(1.0, __dmul_rn(__ddiv_rn(y, (double)j), e));
    for (int i = 0; i < 10; i++) e = __dmul_rn(e, e);
    return e;
#else
    double y = -t / 1024.0;
    double e = 1.0;
    for (int j = 12; j >= 1; j--) e = 1.0 + (y / (double)j) * e;
    for (int i = 0; i < 10; i++) e = e * e;
    return e;
#endif
}

}  // namespace tsz
