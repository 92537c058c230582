// tsz_decompress.cu -- decompression kernels (Section IV-B of arXiv 2602.17552).
//
//   k_parse_header   one thread: validate the stream header against the call
//                    and the buffer size, fill the control block; with the
//                    literal-interpolation flag the CTA then solves for the
//                    RBF weights
//   k_dec_tile_*     offset pre-pass: per 8192-point tile, payload words and
//                    extremum counts -> exclusive prefixes (MD^ bookkeeping)
//   k_decode_ranks   the inverse codec on the rank stream (delta sequence)
//   k_decode_fused   persistent wavefront over tiles: BE^, LZ^ + B^, QZ^ (planes
//                    unpacked with warp shuffles, inverse Lorenzo by a warp
//                    prefix sum), then CP^ + RP^ extrema stencils evaluated on
//                    the QZ^ snapshot and applied, then the lost saddles
//                    collected -- each stage trailing the previous one by the
//                    neighbour reach, so the field stays in L2 in between
//   k_saddle_rounds  cooperative RS^ colour rounds (evaluate, grid sync, write)
// Every read of the stream is bounds-checked against the validated header; a
// violation sets CORRUPT_STREAM and skips the access.
#include <cooperative_groups.h>

#include "tsz_internal.h"

namespace cg = cooperative_groups;

namespace tsz {

// Decode tiles of the fused decoder: 256 blocks (8192 points), 8 warps with
// one block per lane.
constexpr int DT_WARPS = 8;
constexpr int DT_BLOCKS = DT_WARPS * 32;

// The decoder's tiles: linear tiles of 8192 points (labels, extremum lists,
// the wavefront) and payload tiles of 256 blocks.  In format v1 they are the
// same tiles; in format v2 the per-tile counts and prefixes cover the larger
// number of the two.
__host__ __device__ inline uint32_t lin_tiles(const Geo& g) {
    return (uint32_t)((g.n + (uint64_t)DT_BLOCKS * 32 - 1) / ((uint64_t)DT_BLOCKS * 32));
}
__host__ __device__ inline uint32_t all_tiles(const Geo& g) {
    return hmax<uint32_t>(lin_tiles(g), (g.nb + DT_BLOCKS - 1) / DT_BLOCKS);
}

// Label word wi with the codes of points >= n cleared (a valid stream has
// them zero already; clearing keeps every count consistent on any stream).
__device__ __forceinline__ uint32_t label_word(const uint32_t* labels, uint32_t wi, uint32_t n) {
    const uint32_t nwords = (n + 15) / 16;
    if (wi >= nwords) return 0u;
    uint32_t w = __ldg(labels + wi);
    const uint32_t first = wi * 16u;
    if (first + 16u > n) w &= (1u << (2u * (n - first))) - 1u;
    return w;
}

template <class T>
__device__ __forceinline__ T get(const uint8_t* h, int off) {
    return *reinterpret_cast<const T*>(h + off);
}

__device__ void parse_header(const uint8_t* in, uint64_t in_size, uint64_t n_out, Ctrl* c, int* status,
                             uint32_t test_hold) {
    const uint32_t version = in_size >= HDR ? get<uint32_t>(in, 4) : 0u;
    if (in_size < HDR || get<uint32_t>(in, 0) != MAGIC || (version != VERSION && version != VERSION_TILES) ||
        get<uint32_t>(in, 12) != L) {
        set_status(status, ST_CORRUPT);
        return;
    }
    const bool tiles = version == VERSION_TILES;
    const int ndim = (int)get<uint32_t>(in, 8);
    const uint64_t nx = get<uint64_t>(in, 16), ny = get<uint64_t>(in, 24), nz = get<uint64_t>(in, 32);
    const uint32_t flags = get<uint32_t>(in, 40);
    bool ok = (ndim == 2 || ndim == 3) && nx >= 1 && ny >= 1 && nz >= 1 && nx < (1ull << 31) &&
              ny < (1ull << 31) && nz < (1ull << 31) && (ndim == 3 || nz == 1) &&
              flags <= (FLAG_NO_TOPO | FLAG_RBF_SOLVE);
    const uint64_t n = ok ? nx * ny : 0;
    ok = ok && n < (1ull << 31) && n * nz < (1ull << 31) && n * nz == n_out && get<uint64_t>(in, 104) == n_out;
    const uint64_t nb = get<uint64_t>(in, 112);
    ok = ok && nb == (tiles ? tile_blocks(ndim, nx, ny, nz) : cdiv(n_out, L));
    const float w_f = get<float>(in, 64), h_f = get<float>(in, 72);
    const int32_t rk = (int32_t)get<uint32_t>(in, 88);
    const uint32_t sweeps = get<uint32_t>(in, 96);
    const uint64_t kmin = get<uint64_t>(in, 120), kmax = get<uint64_t>(in, 128);
    const uint64_t pay = get<uint64_t>(in, 208), rpay = get<uint32_t>(in, 216);
    const float sigma = get<float>(in, 92);
    const bool topo = !(flags & FLAG_NO_TOPO);
    ok = ok && isfinite(w_f) && w_f > 0.0f && isfinite(h_f) && h_f >= 0.0f;
    ok = ok && (!(flags & FLAG_RBF_SOLVE) || (isfinite(sigma) && sigma > 0.0f));
    ok = ok && (rk == 3 || rk == 5 || rk == 7) && sweeps >= 1 && sweeps <= 16;
    ok = ok && kmin <= cdiv(n_out, 2) && kmax <= cdiv(n_out, 2) && (topo || (kmin == 0 && kmax == 0));
    ok = ok && pay <= nb * (L + 1) && rpay <= cdiv(kmin + kmax, L) * (L + 1);
    if (!ok) {
        set_status(status, ST_CORRUPT);
        return;
    }
    Layout lo;
    make_layout(n_out, nb, topo, pay, kmin + kmax, rpay, lo);
    if (lo.end != get<uint64_t>(in, 200) || lo.end > in_size || lo.s1 != get<uint64_t>(in, 152) ||
        lo.s2 != get<uint64_t>(in, 160) || lo.s4 != get<uint64_t>(in, 168) ||
        lo.s6 != get<uint64_t>(in, 176) || lo.s5 != get<uint64_t>(in, 184) ||
        (topo ? lo.s7 : lo.end) != get<uint64_t>(in, 192)) {
        set_status(status, ST_CORRUPT);
        return;
    }
    Geo g;
    g.ndim = ndim;
    g.nx = (uint32_t)nx;
    g.ny = (uint32_t)ny;
    g.nz = (uint32_t)nz;
    g.n = (uint32_t)n_out;
    g.nxy = (uint32_t)(nx * ny);
    g.nb = (uint32_t)nb;
    geo_divs(g);
    c->g = g;
    c->flags = flags | (tiles ? FLAG_TILE_BLOCKS : 0u);
    c->nb_fmt = (uint32_t)nb;
    c->w_f = w_f;
    c->h_f = h_f;
    c->rbf_k = rk;
    c->rbf_sigma = sigma;
    c->rs_sweeps = (int)sweeps;
    c->pay_words = pay;
    c->rank_words = rpay;
    c->k_total = kmin + kmax;
    c->lo = lo;
    c->test_hold = test_hold;
    for (int i = 0; i < 9; i++) c->g_rbf[i] = get<float>(in, 220 + 4 * i);
}

// Weights of the literal RBF interpolation (Section IV-B(3), Eqs.
// RBF-interp-final and RBF-eval) at p for the nodes q_i of N_r(p) \ {p} in
// (z, y, x) table order: the Gaussian interpolant with a constant term,
// s(x) = sum_i w_i phi(|x - q_i|) + c with sum_i w_i = 0, which reproduces
// constants, so the weights sum to one as Eq. RBF-eval states.  With
// a = Phi^-1 phi_p and b = Phi^-1 1 the weights are a + b (1 - sum a) / sum b.
// One CTA, binary64 without contraction.  Phi = L L^T by right-looking
// Cholesky: column j is finished (square root, division), then the trailing
// triangle loses column j's products, so every entry sees its subtractions
// in ascending column order -- the operations and their order of the
// textbook column-by-column factorisation.  Substitutions the same way
// (forward: ascending, back: descending).  Phi's entries depend on the
// squared node distance only (0 .. 4 r^2): one exp per distinct distance.
__device__ void rbf_solve_block(int ndim, int r, float sigma, float* alpha, double* sm) {
    __shared__ int s_d2[RBF_MAX_NODES], s_x[RBF_MAX_NODES], s_y[RBF_MAX_NODES], s_z[RBF_MAX_NODES];
    __shared__ double s_phi[37];
    __shared__ int s_m;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        const int rz = ndim == 3 ? r : 0;
        int m = 0;
        for (int dz = -rz; dz <= rz; dz++)
            for (int dy = -r; dy <= r; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    const int d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 == 0 || d2 > r * r) continue;
                    s_x[m] = dx, s_y[m] = dy, s_z[m] = dz, s_d2[m] = d2;
                    m++;
                }
        s_m = m;
    }
    const double s = (double)sigma;
    const double s2 = __dmul_rn(__dmul_rn(2.0, s), s);
    for (int d = tid; d <= 4 * r * r; d += nt) s_phi[d] = exp_neg(__ddiv_rn((double)d, s2));
    __syncthreads();
    const int m = s_m;
    double* A = sm;            // m x m row-major; the lower triangle holds Phi, then L
    double* X = sm + m * m;    // two right-hand sides (phi_p, ones), then the solutions
    for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx / m, j = idx - i * m;
        if (j > i) continue;
        const int a = s_x[i] - s_x[j], b = s_y[i] - s_y[j], cz = s_z[i] - s_z[j];
        A[idx] = s_phi[a * a + b * b + cz * cz];
    }
    for (int i = tid; i < m; i += nt) {
        X[i] = s_phi[s_d2[i]];
        X[m + i] = 1.0;
    }
    __syncthreads();
    for (int j = 0; j < m; j++) {
        if (tid == 0) A[j * m + j] = __dsqrt_rn(A[j * m + j]);
        __syncthreads();
        for (int i = j + 1 + tid; i < m; i += nt) A[i * m + j] = __ddiv_rn(A[i * m + j], A[j * m + j]);
        __syncthreads();
        const int t = m - 1 - j;
        for (int idx = tid; idx < t * t; idx += nt) {
            const int i = j + 1 + idx / t, k = j + 1 + idx % t;
            if (k > i) continue;
            A[i * m + k] = __dsub_rn(A[i * m + k], __dmul_rn(A[i * m + j], A[k * m + j]));
        }
        __syncthreads();
    }
    for (int i = 0; i < m; i++) {   // L y = rhs
        if (tid < 2) X[tid * m + i] = __ddiv_rn(X[tid * m + i], A[i * m + i]);
        __syncthreads();
        const int t = m - 1 - i;
        for (int idx = tid; idx < 2 * t; idx += nt) {
            const int h = idx / t, i2 = i + 1 + idx % t;
            X[h * m + i2] = __dsub_rn(X[h * m + i2], __dmul_rn(A[i2 * m + i], X[h * m + i]));
        }
        __syncthreads();
    }
    for (int i = m - 1; i >= 0; i--) {   // L^T x = y
        if (tid < 2) X[tid * m + i] = __ddiv_rn(X[tid * m + i], A[i * m + i]);
        __syncthreads();
        for (int idx = tid; idx < 2 * i; idx += nt) {
            const int h = idx / i, i2 = idx % i;
            X[h * m + i2] = __dsub_rn(X[h * m + i2], __dmul_rn(A[i * m + i2], X[h * m + i]));
        }
        __syncthreads();
    }
    if (tid == 0) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < m; i++) sa = __dadd_rn(sa, X[i]);
        for (int i = 0; i < m; i++) sb = __dadd_rn(sb, X[m + i]);
        const double cf = __ddiv_rn(__dsub_rn(1.0, sa), sb);
        for (int i = 0; i < m; i++) alpha[i] = __double2float_rn(__dadd_rn(X[i], __dmul_rn(X[m + i], cf)));
    }
}

// bytes of dynamic shared memory rbf_solve_block() takes at most
constexpr int RBF_SOLVE_SMEM = (RBF_MAX_NODES * RBF_MAX_NODES + 2 * RBF_MAX_NODES) * 8;

__global__ void __launch_bounds__(256) k_parse_header(const uint8_t* in, uint64_t in_size, uint64_t n_out,
                                                      Ctrl* c, int* status, uint32_t test_hold) {
    griddep_enter();
    extern __shared__ double sm_solve[];
    __shared__ int s_solve;
    if (threadIdx.x == 0) {
        parse_header(in, in_size, n_out, c, status, test_hold);
        s_solve = *status == 0 && (c->flags & (FLAG_NO_TOPO | FLAG_RBF_SOLVE)) == FLAG_RBF_SOLVE;
    }
    __syncthreads();
    if (s_solve) rbf_solve_block(c->g.ndim, c->rbf_k / 2, c->rbf_sigma, c->rbf_alpha, sm_solve);
}

// --------------------------------------------------------------- inverse codec

// Decode one block held by a warp: lanes 0..w load the sign plane and the w
// magnitude planes; each lane rebuilds its residual from the broadcast planes,
// a warp prefix sum undoes the Lorenzo step.  Unsigned arithmetic keeps a
// corrupt stream from invoking signed overflow.
__device__ __forceinline__ int32_t decode_block(const uint32_t* pay, unsigned long long woff, uint32_t w,
                                                int32_t first, int lane) {
    uint32_t word = (lane <= (int)w) ? pay[woff + lane] : 0u;
    uint32_t sgn = (__shfl_sync(FULL, word, 0) >> lane) & 1u;
    uint32_t mag = 0;
    for (uint32_t p = 0; p < w; p++) mag |= ((__shfl_sync(FULL, word, p + 1) >> lane) & 1u) << p;
    uint32_t d = sgn ? 0u - mag : mag;
    if (lane == 0) d = 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, d, o);
        if (lane >= o) d += t;
    }
    return (int32_t)((uint32_t)first + d);
}

// Rank-sequence decoder (BE^, LZ^ + B^ on the delta sequence): 8192-delta
// tiles with payload offsets from the pre-pass, one block per thread (the
// field decoder's scheme), output through a padded shared buffer.
__global__ void __launch_bounds__(256, 3) k_decode_ranks(const uint8_t* __restrict__ in, Ctrl* c,
                                                         const uint32_t* rpre, int32_t* __restrict__ delta,
                                                         int* status) {
    griddep_enter();
    __shared__ __align__(16) uint32_t s_buf[DT_BLOCKS * 36];
    __shared__ uint32_t s_w[8];
    if (*status || (c->flags & FLAG_NO_TOPO)) return;
    const Layout lo = c->lo;
    const uint64_t k = c->k_total;
    const unsigned long long rwords = c->rank_words;
    const uint32_t nbd = (uint32_t)cdiv(k, L);
    const uint32_t nrt = (nbd + DT_BLOCKS - 1) / DT_BLOCKS;
    const uint8_t* widths = in + lo.r2;
    const int32_t* firsts = reinterpret_cast<const int32_t*>(in + lo.r4);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(in + lo.r5);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool corrupt = false;
    for (uint32_t t = blockIdx.x; t < nrt; t += gridDim.x) {
        const uint32_t P0 = rpre[t], P1 = rpre[t + 1];
        uint32_t len = 0;
        if (P1 >= P0 && P1 - P0 <= DT_BLOCKS * 33u && P1 <= rwords) len = P1 - P0;
        else corrupt = true;
        const uint32_t b = t * DT_BLOCKS + threadIdx.x;
        uint32_t w = 0;
        int32_t f = 0;
        if (b < nbd) {   // issued before the payload loads: both in flight together
            w = __ldg(widths + b);
            f = __ldg(firsts + b);
        }
        for (uint32_t i0 = 0; i0 < len; i0 += 4 * DT_BLOCKS) {   // four loads in flight per thread
            uint32_t v4[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t i = i0 + j * DT_BLOCKS + threadIdx.x;
                v4[j] = i < len ? __ldg(pay + P0 + i) : 0u;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t i = i0 + j * DT_BLOCKS + threadIdx.x;
                if (i < len) s_buf[i] = v4[j];
            }
        }
        if (w > 32) w = 0;
        const uint32_t words = w ? 1u + w : 0u;
        uint32_t iw = words;
#pragma unroll
        for (int of = 1; of < 32; of <<= 1) {
            const uint32_t a0 = __shfl_up_sync(FULL, iw, of);
            if (lane >= (uint32_t)of) iw += a0;
        }
        if (lane == 31) s_w[warp] = iw;
        __syncthreads();
        uint32_t woff = iw - words;
        for (uint32_t q = 0; q < warp; q++) woff += s_w[q];
        uint32_t v[32];
        uint32_t sgn = 0;
        uint32_t wv = w;   // planes present (0: constant block or a damaged stream)
        if (w && woff + 1 + w > len) {
            corrupt = true;
            wv = 0;
        }
        if (wv) sgn = s_buf[woff];
        planes_to_values(__reduce_max_sync(FULL, wv), wv, [&](int r) { return s_buf[woff + 1 + r]; }, v);
        {
            int32_t q = f;
#pragma unroll
            for (int e = 0; e < 32; e++) {
                if (e) q += (sgn >> e) & 1u ? -(int32_t)v[e] : (int32_t)v[e];
                v[e] = (uint32_t)q;
            }
        }
        __syncthreads();   // the payload is consumed: the buffer stages the output rows
        {
            uint32_t* row = s_buf + threadIdx.x * 36;
#pragma unroll
            for (int q = 0; q < 8; q++)
                *reinterpret_cast<uint4*>(row + 4 * q) = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        __syncthreads();
        const uint64_t p0 = (uint64_t)t * (DT_BLOCKS * 32);
        const uint64_t left = k - p0;
        const uint32_t np = left < (uint64_t)(DT_BLOCKS * 32) ? (uint32_t)left : (uint32_t)(DT_BLOCKS * 32);
        for (uint32_t i = threadIdx.x; i < np; i += blockDim.x)
            delta[p0 + i] = (int32_t)s_buf[(i >> 5) * 36 + (i & 31)];
        __syncthreads();
    }
    if (corrupt) set_status(status, ST_CORRUPT);
}

// ------------------------------------------------------------- fix-up stages

// Move x by kk representable binary32 values on the ordered-integer line
// ("delta * eta" with eta the machine epsilon of x's binade).  False if the
// result would not be finite.
__device__ __forceinline__ bool step_ulps(float x, long long kk, float& res) {
    uint32_t b = __float_as_uint(x);
    long long o = (b & 0x80000000u) ? -(long long)(b & 0x7FFFFFFFu) : (long long)b;
    o += kk;
    if (o >= 0x7F800000ll || o <= -0x7F800000ll) return false;
    uint32_t nb = o >= 0 ? (uint32_t)o : (0x80000000u | (uint32_t)(-o));
    res = __uint_as_float(nb);
    return true;
}

struct OverrideVal {   // the field with point p set to v
    const float* F;
    uint32_t p;
    float v;
    __device__ __forceinline__ float operator()(uint32_t j) const { return j == p ? v : F[j]; }
};

__device__ __forceinline__ int colour_of(const Geo& g, uint32_t x, uint32_t y, uint32_t z) {
    return g.ndim == 2 ? (int)((x + 2u * y) % 5u) : (int)((x + 2u * y + 3u * z) % 7u);
}

// Offsets of the RBF neighbourhood N_r(p) \ {p} in the fixed (z, y, x)
// ascending order, with their squared length; built per CTA in shared memory.
struct RbfTable {
    int n;                 // number of offsets
    float den_full;        // sum of the weights in table order (all in the domain)
    int dx[122], dy[122], dz[122], d2[122];
    int lin[122];          // linear offset dx + dy nx + dz nx ny
};

__device__ void build_rbf_table(RbfTable& T, const Geo& g, const Ctrl* c) {
    if (threadIdx.x == 0) {
        const int r = c->rbf_k / 2, rz = g.ndim == 3 ? r : 0;
        int m = 0;
        float den = 0.0f;
        for (int dz = -rz; dz <= rz; dz++)
            for (int dy = -r; dy <= r; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    const int d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 == 0 || d2 > r * r) continue;
                    T.dx[m] = dx;
                    T.dy[m] = dy;
                    T.dz[m] = dz;
                    T.d2[m] = d2;
                    T.lin[m] = dx + dy * (int)g.nx + dz * (int)g.nxy;
                    den = __fadd_rn(den, c->g_rbf[d2 - 1]);
                    m++;
                }
        T.n = m;
        T.den_full = den;
    }
    __syncthreads();
}

// Relation of a neighbour value u to p once p moves by a step smaller than
// half the smallest nonzero gap: distinct neighbours keep their side, ties go
// to the side opposite the move (up: tie -> lower).
__device__ __forceinline__ bool higher_after(float u, float fp, bool up) { return u > fp || (u == fp && !up); }
__device__ __forceinline__ bool lower_after(float u, float fp, bool up) { return u < fp || (u == fp && up); }

// Could some small move of p (up or down) make it a saddle, given its face
// neighbours nb[0..2*ndim)?  (RS^ check (a) over every admissible step.)
__device__ __forceinline__ bool saddle_feasible(const float* nb, int ndim, float fp) {
    bool any = false;
#pragma unroll
    for (int up = 0; up < 2; up++) {
        int ph = 0, pl = 0, px = 0;
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
            if (ax >= ndim) break;
            const float a = nb[2 * ax], b = nb[2 * ax + 1];
            if (higher_after(a, fp, up) && higher_after(b, fp, up)) ph++;
            else if (lower_after(a, fp, up) && lower_after(b, fp, up)) pl++;
            else px++;
        }
        any |= px == 0 && ph > 0 && pl > 0;
    }
    return any;
}

// RS^ candidate: returns true and the refined value when accepted.  Runs only
// inside the cooperative rounds kernel, whose grid syncs order every write of
// the previous colour before these (L1-cached) reads.
__device__ bool saddle_candidate(const float* F, const uint32_t* labels, const Geo& g, const Ctrl* c,
                                 const RbfTable& T, uint32_t p, uint32_t x, uint32_t y, uint32_t z, float& vout) {
    // a saddle label is only valid at interior points; anything else is a bad stream
    if (x == 0 || x + 1 >= g.nx || y == 0 || y + 1 >= g.ny || (g.ndim == 3 && (z == 0 || z + 1 >= g.nz)))
        return false;
    const float Fp = F[p];
    const uint32_t st[3] = {1u, g.nx, g.nxy};
    float nb[6];
    for (int ax = 0; ax < g.ndim; ax++) {
        nb[2 * ax] = F[p - st[ax]];
        nb[2 * ax + 1] = F[p + st[ax]];
    }
    // current type: s means the saddle is not lost (any more)
    {
        int ph = 0, pl = 0, px = 0;
        for (int ax = 0; ax < g.ndim; ax++) {
            const float a = nb[2 * ax], b = nb[2 * ax + 1];
            if (a > Fp && b > Fp) ph++;
            else if (a < Fp && b < Fp) pl++;
            else px++;
        }
        if (px == 0 && ph > 0 && pl > 0) return false;
    }
    float gmin = __int_as_float(0x7F800000);
    for (int i = 0; i < 2 * g.ndim; i++) {
        const float gi = fabsf(__fsub_rn(nb[i], Fp));
        if (gi > 0.0f && gi < gmin) gmin = gi;
    }
    if (isinf(gmin)) return false;
    const bool solve = c->flags & FLAG_RBF_SOLVE;
    // Exact shortcut: |v - Fp| <= gmin / 2 keeps every distinct neighbour on its
    // side, so p's type with v depends only on the direction of the move; if
    // neither direction gives a saddle, check (a) below rejects every v.  (The
    // unclamped literal interpolation can step further: no shortcut there.)
    if (!solve && !saddle_feasible(nb, g.ndim, Fp)) return false;
    // normalised Gaussian kernel over N_r(p) \ {p}, fixed (z, y, x) order; with
    // the literal interpolation and the ball inside the grid, the
    // interpolant's value at p instead: sum alpha_e F(p + o_e)
    const int r = c->rbf_k / 2;
    const bool inside = x >= (uint32_t)r && x + r < g.nx && y >= (uint32_t)r && y + r < g.ny &&
                        (g.ndim == 2 || (z >= (uint32_t)r && z + r < g.nz));
    float num = 0.0f, den;
    if (inside && solve) {
#pragma unroll 8
        for (int e = 0; e < T.n; e++) num = __fadd_rn(num, __fmul_rn(c->rbf_alpha[e], F[(int)p + T.lin[e]]));
        den = 1.0f;
    } else if (inside) {
#pragma unroll 8
        for (int e = 0; e < T.n; e++) num = __fadd_rn(num, __fmul_rn(c->g_rbf[T.d2[e] - 1], F[(int)p + T.lin[e]]));
        den = T.den_full;
    } else {
        den = 0.0f;
        for (int e = 0; e < T.n; e++) {
            const long long xx = (long long)x + T.dx[e], yy = (long long)y + T.dy[e], zz = (long long)z + T.dz[e];
            if (xx < 0 || yy < 0 || zz < 0 || xx >= g.nx || yy >= g.ny || zz >= g.nz) continue;
            const float gw = c->g_rbf[T.d2[e] - 1];
            num = __fadd_rn(num, __fmul_rn(gw, F[(int)p + T.lin[e]]));
            den = __fadd_rn(den, gw);
        }
    }
    const float u = inside && solve ? num : __fdiv_rn(num, den);
    float v = u;   // the literal interpolation: unclamped, acceptance alone bounds the step
    if (!solve) {
        const float capv = fminf(__fmul_rn(0.1f, c->h_f), __fmul_rn(0.5f, gmin));
        float stp = __fsub_rn(u, Fp);
        if (stp > capv) stp = capv;
        if (stp < -capv) stp = -capv;
        v = __fadd_rn(Fp, stp);
    }
    if (v == Fp) return false;
    GlobalVal val{F};
    OverrideVal nv{F, p, v};
    if (classify_interior(nv, g, p, v) != LAB_SAD) return false;   // (a): p is interior
    for (int ax = 0; ax < g.ndim; ax++) {                          // (b)
        for (int sg = -1; sg <= 1; sg += 2) {
            const uint32_t q = sg < 0 ? p - st[ax] : p + st[ax];
            // q's type depends on p only through p's order against f(q)
            const float fq0 = F[q];
            if ((v > fq0) == (Fp > fq0) && (v < fq0) == (Fp < fq0)) continue;
            uint32_t qx = x, qy = y, qz = z;
            if (ax == 0) qx = sg < 0 ? x - 1 : x + 1;
            else if (ax == 1) qy = sg < 0 ? y - 1 : y + 1;
            else qz = sg < 0 ? z - 1 : z + 1;
            const float fq = F[q];
            const int tn = classify_any(nv, g, q, qx, qy, qz, fq);
            const int to = classify_any(val, g, q, qx, qy, qz, fq);
            if (tn != to && tn != label_at(labels, q)) return false;
        }
    }
    if (!(fabsf(__fsub_rn(v, Fp)) <= c->h_f)) return false;       // (c)
    vout = v;
    return true;
}

// ------------------------------------------------- saddle neighbourhood records
//
// Every colour round reads each candidate's RBF neighbourhood.  Read from the
// field, a round's candidates touch about half of its sectors, once per
// colour.  Instead the rounds kernel first copies, in one pass in list order
// (consecutive candidates are neighbours in space, so the copy streams through
// L2), the neighbourhood of every candidate into a compact record stored in
// its colour bucket.  A round then streams its records.  Points that can
// change during the rounds are the listed candidates, all saddle-labelled; the
// record marks the saddle-labelled slots and those are read from the field
// when a round needs them, so a record always gives current values and the
// arithmetic is exactly that of saddle_candidate().  Every candidate gets a
// record, also near the grid's faces, where a mask marks the slots inside the
// grid: field reads there would make the few warps holding such a candidate
// two to three times slower, and those warps set the end of every round.
//
// Slots: the RBF neighbourhood N_r(p) \ {p} in the RBF table's (z, y, x)
// order, then the remaining points at Manhattan distance 1..2 (the face
// neighbours and their face neighbours, read by checks (a) and (b)).

template <int ND, int R>
struct RecStencil {
    int ns = 0, n = 0;   // RBF slots, all slots (<= 32)
    int dx[32] = {}, dy[32] = {}, dz[32] = {}, d2[32] = {};
    int face[6] = {};    // slot of p's face neighbour f, order (x-, x+, y-, y+, z-, z+)
    int nbr[6][6] = {};  // slot of face neighbour k of face neighbour f; -1: p itself
    __host__ __device__ constexpr int find(int x, int y, int z) const {
        for (int i = 0; i < n; i++)
            if (dx[i] == x && dy[i] == y && dz[i] == z) return i;
        return -1;
    }
    __host__ __device__ constexpr RecStencil() {
        const int rz = ND == 3 ? R : 0;
        for (int z = -rz; z <= rz; z++)
            for (int y = -R; y <= R; y++)
                for (int x = -R; x <= R; x++) {
                    const int q = x * x + y * y + z * z;
                    if (q == 0 || q > R * R) continue;
                    dx[n] = x, dy[n] = y, dz[n] = z, d2[n] = q;
                    n++;
                }
        ns = n;
        const int z2 = ND == 3 ? 2 : 0;
        for (int z = -z2; z <= z2; z++)
            for (int y = -2; y <= 2; y++)
                for (int x = -2; x <= 2; x++) {
                    const int m = (x < 0 ? -x : x) + (y < 0 ? -y : y) + (z < 0 ? -z : z);
                    if (m == 0 || m > 2 || find(x, y, z) >= 0) continue;
                    dx[n] = x, dy[n] = y, dz[n] = z, d2[n] = x * x + y * y + z * z;
                    n++;
                }
        for (int f = 0; f < 2 * ND; f++) {
            const int ax = f / 2, sg = f % 2 ? 1 : -1;
            const int fx = ax == 0 ? sg : 0, fy = ax == 1 ? sg : 0, fz = ax == 2 ? sg : 0;
            face[f] = find(fx, fy, fz);
            for (int k = 0; k < 2 * ND; k++) {
                const int bx = k / 2, bs = k % 2 ? 1 : -1;
                const int gx = fx + (bx == 0 ? bs : 0), gy = fy + (bx == 1 ? bs : 0), gz = fz + (bx == 2 ? bs : 0);
                nbr[f][k] = (gx == 0 && gy == 0 && gz == 0) ? -1 : find(gx, gy, gz);
            }
        }
    }
    // the slots of the RBF neighbourhood, and face f's neighbours (p is always inside)
    __host__ __device__ constexpr uint32_t ball_mask() const { return ns == 32 ? 0xFFFFFFFFu : (1u << ns) - 1u; }
    __host__ __device__ constexpr uint32_t nbr_mask(int f) const {
        uint32_t m = 0;
        for (int k = 0; k < 2 * ND; k++)
            if (nbr[f][k] >= 0) m |= 1u << nbr[f][k];
        return m;
    }
    // record words: the slots, the saddle-slot mask and the in-grid mask, padded to 16 bytes
    __host__ __device__ constexpr int words() const { return (n + 2 + 3) / 4 * 4; }
};
constexpr int REC_MAX_WORDS = 36;   // the largest record (3D, r = 2)
static_assert(RecStencil<3, 1>{}.words() <= REC_MAX_WORDS && RecStencil<3, 2>{}.words() <= REC_MAX_WORDS &&
                  RecStencil<2, 1>{}.words() <= REC_MAX_WORDS && RecStencil<2, 2>{}.words() <= REC_MAX_WORDS &&
                  RecStencil<2, 3>{}.words() <= REC_MAX_WORDS,
              "record size");
static_assert(RecStencil<3, 2>{}.n <= 32 && RecStencil<2, 3>{}.n <= 32, "slot masks are 32 bits");

// Record kinds: 3D r = 1, 2 and 2D r = 1, 2, 3 (3D r = 3 keeps the field reads).
__host__ __device__ inline bool rec_supported(int ndim, int r) {
    return ndim == 3 ? (r == 1 || r == 2) : (r >= 1 && r <= 3);
}

constexpr uint32_t REC_W31 = RecStencil<3, 1>{}.words(), REC_W32 = RecStencil<3, 2>{}.words();
constexpr uint32_t REC_W21 = RecStencil<2, 1>{}.words(), REC_W22 = RecStencil<2, 2>{}.words();
constexpr uint32_t REC_W23 = RecStencil<2, 3>{}.words();
// words of one record of a supported kind (at most REC_MAX_WORDS): the
// records are packed at this stride, so that they fill whole sectors
__host__ __device__ inline uint32_t rec_words(int ndim, int r) {
    if (ndim == 3) return r == 1 ? REC_W31 : REC_W32;
    return r == 1 ? REC_W21 : r == 2 ? REC_W22 : REC_W23;
}

// Candidates whose whole RBF neighbourhood and both face rings lie inside the
// grid: their record has every slot (no bounds checks when it is gathered).
__device__ __forceinline__ bool rec_inside(const Geo& g, int r, uint32_t x, uint32_t y, uint32_t z) {
    const uint32_t m = r > 2 ? (uint32_t)r : 2u;
    return x >= m && x + m < g.nx && y >= m && y + m < g.ny && (g.ndim == 2 || (z >= m && z + m < g.nz));
}

// A candidate's record: its slot values, the saddle-labelled slots (read live
// in the rounds) and the slots inside the grid.  Near the grid's faces some
// slots lie outside: they are not read and their bit is clear.
template <int ND, int R>
__device__ __forceinline__ void rec_gather(const float* F, const uint32_t* labels, const Geo& g, uint32_t p,
                                           uint32_t x, uint32_t y, uint32_t z, bool inside, uint32_t* rec) {
    constexpr RecStencil<ND, R> S{};
    constexpr int W = S.words();
    uint32_t w[W];
    uint32_t dyn = 0, vm = 0;
#pragma unroll
    for (int e = 0; e < S.n; e++) {
        const bool in = inside || ((long long)x + S.dx[e] >= 0 && (long long)x + S.dx[e] < (long long)g.nx &&
                                   (long long)y + S.dy[e] >= 0 && (long long)y + S.dy[e] < (long long)g.ny &&
                                   (long long)z + S.dz[e] >= 0 && (long long)z + S.dz[e] < (long long)g.nz);
        uint32_t wv = 0u;
        if (in) {
            const uint32_t q = p + (uint32_t)(S.dx[e] + S.dy[e] * (int)g.nx + S.dz[e] * (int)g.nxy);
            wv = __float_as_uint(F[q]);
            dyn |= (label_at(labels, q) == LAB_SAD ? 1u : 0u) << e;
            vm |= 1u << e;
        }
        w[e] = wv;
    }
    w[S.n] = dyn;
    w[S.n + 1] = vm;
#pragma unroll
    for (int e = S.n + 2; e < W; e++) w[e] = 0u;
    uint4* d = reinterpret_cast<uint4*>(rec);
#pragma unroll
    for (int k = 0; k < W / 4; k++) d[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
}

// classify_interior()'s rule on explicit values: centre v, face neighbours n[]
template <int ND>
__device__ __forceinline__ int cls_vals(float v, const float* n) {
    const bool Hx = n[0] > v && n[1] > v, Lx = n[0] < v && n[1] < v;
    const bool Hy = n[2] > v && n[3] > v, Ly = n[2] < v && n[3] < v;
    const bool Hz = ND != 3 || (n[4] > v && n[5] > v), Lz = ND != 3 || (n[4] < v && n[5] < v);
    const bool m = Hx && Hy && Hz, M = Lx && Ly && Lz;
    const bool s = (Hx || Lx) && (Hy || Ly) && (Hz || Lz) && !m && !M;
    return (int)((uint32_t)(m | M) | ((uint32_t)(s | M) << 1));
}

// classify()'s rule for a point with a face neighbour outside the grid
// (present: bit k set for neighbour k): a minimum or maximum over the
// neighbours present, never a saddle.
template <int ND>
__device__ __forceinline__ int cls_vals_cut(float v, const float* n, uint32_t present) {
    int nn = 0, nhi = 0, nlo = 0;
#pragma unroll
    for (int k = 0; k < 2 * ND; k++) {
        if (!((present >> k) & 1u)) continue;
        nn++;
        nhi += n[k] > v;
        nlo += n[k] < v;
    }
    if (nn == 0) return LAB_R;
    return nhi == nn ? LAB_MIN : (nlo == nn ? LAB_MAX : LAB_R);
}

// saddle_candidate() for a candidate with a record: the same arithmetic in the
// same order.  Slots outside the grid (clear bits of the record's in-grid
// mask) are never read: a cut RBF ball takes the normalised kernel over the
// slots inside, a face neighbour on the grid's boundary is classified over
// the neighbours it has.
template <int ND, int R>
__device__ bool saddle_candidate_rec(const float* F, const uint32_t* labels, const Geo& g, const Ctrl* c,
                                     float den_full, uint32_t p, const uint32_t* rec, float& vout) {
    constexpr RecStencil<ND, R> S{};
    constexpr int W = S.words();
    uint32_t w[W];
    const uint4* s4 = reinterpret_cast<const uint4*>(rec);
#pragma unroll
    for (int k = 0; k < W / 4; k++) {
        const uint4 t = s4[k];
        w[4 * k] = t.x, w[4 * k + 1] = t.y, w[4 * k + 2] = t.z, w[4 * k + 3] = t.w;
    }
    const uint32_t dyn = w[S.n], vm = w[S.n + 1];
    // a saddle label is only valid at interior points; anything else is a bad stream
#pragma unroll
    for (int f = 0; f < 2 * ND; f++)
        if (!((vm >> S.face[f]) & 1u)) return false;
    float v[S.n];
#pragma unroll
    for (int e = 0; e < S.n; e++)
        v[e] = (dyn >> e) & 1u ? F[p + (uint32_t)(S.dx[e] + S.dy[e] * (int)g.nx + S.dz[e] * (int)g.nxy)]
                               : __uint_as_float(w[e]);
    const float Fp = F[p];
    float nb[2 * ND];
#pragma unroll
    for (int f = 0; f < 2 * ND; f++) nb[f] = v[S.face[f]];
    {
        int ph = 0, pl = 0, px = 0;
#pragma unroll
        for (int ax = 0; ax < ND; ax++) {
            const float a = nb[2 * ax], b = nb[2 * ax + 1];
            if (a > Fp && b > Fp) ph++;
            else if (a < Fp && b < Fp) pl++;
            else px++;
        }
        if (px == 0 && ph > 0 && pl > 0) return false;
    }
    float gmin = __int_as_float(0x7F800000);
#pragma unroll
    for (int i = 0; i < 2 * ND; i++) {
        const float gi = fabsf(__fsub_rn(nb[i], Fp));
        if (gi > 0.0f && gi < gmin) gmin = gi;
    }
    if (isinf(gmin)) return false;
    const bool solve = c->flags & FLAG_RBF_SOLVE;
    if (!solve && !saddle_feasible(nb, ND, Fp)) return false;
    const bool ball_in = (vm & S.ball_mask()) == S.ball_mask();
    float num = 0.0f, vn;
    if (solve && ball_in) {
#pragma unroll
        for (int e = 0; e < S.ns; e++) num = __fadd_rn(num, __fmul_rn(c->rbf_alpha[e], v[e]));
        vn = num;
    } else {
        float den = den_full;
        if (ball_in) {
#pragma unroll
            for (int e = 0; e < S.ns; e++) num = __fadd_rn(num, __fmul_rn(c->g_rbf[S.d2[e] - 1], v[e]));
        } else {   // the ball cut by the grid: its slots inside, in table order
            den = 0.0f;
#pragma unroll
            for (int e = 0; e < S.ns; e++) {
                if (!((vm >> e) & 1u)) continue;
                const float gw = c->g_rbf[S.d2[e] - 1];
                num = __fadd_rn(num, __fmul_rn(gw, v[e]));
                den = __fadd_rn(den, gw);
            }
        }
        const float u = __fdiv_rn(num, den);
        if (solve) {
            vn = u;   // the literal interpolation: unclamped
        } else {
            const float capv = fminf(__fmul_rn(0.1f, c->h_f), __fmul_rn(0.5f, gmin));
            float stp = __fsub_rn(u, Fp);
            if (stp > capv) stp = capv;
            if (stp < -capv) stp = -capv;
            vn = __fadd_rn(Fp, stp);
        }
    }
    if (vn == Fp) return false;
    if (cls_vals<ND>(vn, nb) != LAB_SAD) return false;   // (a)
    const uint32_t st[3] = {1u, g.nx, g.nxy};
#pragma unroll
    for (int f = 0; f < 2 * ND; f++) {                   // (b)
        float qn[2 * ND], qo[2 * ND];
        uint32_t present = 0;
#pragma unroll
        for (int k = 0; k < 2 * ND; k++) {
            const int sl = S.nbr[f][k];
            qn[k] = sl < 0 ? vn : v[sl < 0 ? 0 : sl];
            qo[k] = sl < 0 ? Fp : v[sl < 0 ? 0 : sl];
            present |= (sl < 0 || ((vm >> (sl < 0 ? 0 : sl)) & 1u) ? 1u : 0u) << k;
        }
        const float fq = nb[f];
        // q's type depends on p only through p's order against f(q): if the
        // move keeps it, the type is unchanged (exactly, not as a bound)
        if ((vn > fq) == (Fp > fq) && (vn < fq) == (Fp < fq)) continue;
        int tn, to;
        if (present == (1u << (2 * ND)) - 1u) {
            tn = cls_vals<ND>(fq, qn);
            to = cls_vals<ND>(fq, qo);
        } else {
            tn = cls_vals_cut<ND>(fq, qn, present);
            to = cls_vals_cut<ND>(fq, qo, present);
        }
        if (tn != to) {
            const uint32_t q = f & 1 ? p + st[f >> 1] : p - st[f >> 1];
            if (tn != label_at(labels, q)) return false;
        }
    }
    if (!(fabsf(__fsub_rn(vn, Fp)) <= c->h_f)) return false;   // (c)
    vout = vn;
    return true;
}

// Record dispatch on (ndim, r) (the kinds rec_supported() admits).
__device__ __forceinline__ void rec_gather_any(int ndim, int r, const float* F, const uint32_t* labels,
                                               const Geo& g, uint32_t p, uint32_t x, uint32_t y, uint32_t z,
                                               bool inside, uint32_t* rec) {
    if (ndim == 3) {
        if (r == 1) rec_gather<3, 1>(F, labels, g, p, x, y, z, inside, rec);
        else rec_gather<3, 2>(F, labels, g, p, x, y, z, inside, rec);
    } else {
        if (r == 1) rec_gather<2, 1>(F, labels, g, p, x, y, z, inside, rec);
        else if (r == 2) rec_gather<2, 2>(F, labels, g, p, x, y, z, inside, rec);
        else rec_gather<2, 3>(F, labels, g, p, x, y, z, inside, rec);
    }
}

__device__ __forceinline__ bool saddle_candidate_rec_any(int ndim, int r, const float* F, const uint32_t* labels,
                                                         const Geo& g, const Ctrl* c, float den_full, uint32_t p,
                                                         const uint32_t* rec, float& v) {
    if (ndim == 3) {
        if (r == 1) return saddle_candidate_rec<3, 1>(F, labels, g, c, den_full, p, rec, v);
        return saddle_candidate_rec<3, 2>(F, labels, g, c, den_full, p, rec, v);
    }
    if (r == 1) return saddle_candidate_rec<2, 1>(F, labels, g, c, den_full, p, rec, v);
    if (r == 2) return saddle_candidate_rec<2, 2>(F, labels, g, c, den_full, p, rec, v);
    return saddle_candidate_rec<2, 3>(F, labels, g, c, den_full, p, rec, v);
}

// ---------------------------------------------------------- offset pre-pass
//
// Per decode tile (256 blocks): payload words from the widths and the number of
// extrema (m/M labels) -> exclusive prefixes.  With every tile's offsets known
// up front the fused decoder needs no look-back.

__global__ void __launch_bounds__(256) k_dec_tile_sums(const uint8_t* __restrict__ in, Ctrl* c,
                                                       uint32_t* tile_w, uint32_t* tile_c, uint32_t* rtile_w,
                                                       int* status) {
    griddep_enter();
    // per-slice sums of this CTA's tiles (field words, extrema; rank words),
    // added to the control block once per slice at the end
    __shared__ unsigned long long s_sl[SCAN_SLICES][3];
    for (uint32_t i = threadIdx.x; i < SCAN_SLICES * 3; i += blockDim.x) s_sl[i / 3][i % 3] = 0;
    __syncthreads();
    if (*status) return;
    const Geo g = c->g;
    const Layout lo = c->lo;
    const bool topo = !(c->flags & FLAG_NO_TOPO);
    const uint8_t* widths = in + lo.s2;
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(in + lo.s6);
    const uint32_t ntiles = all_tiles(g);
    const bool tiles = c->flags & FLAG_TILE_BLOCKS;
    const int lane = threadIdx.x & 31;
    bool corrupt = false;
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += (gridDim.x * blockDim.x) >> 5) {
        uint32_t words = 0, cps = 0;
#pragma unroll
        for (int j = 0; j < DT_BLOCKS / 32; j++) {
            const uint32_t b = t * DT_BLOCKS + j * 32 + lane;
            if (b < g.nb) {
                // format v2: bit 7 picks the block's predictor (never with w = 0)
                const uint32_t wb = __ldg(widths + b);
                uint32_t w = tiles ? (wb & 0x7Fu) : wb;
                if (w > 32 || (tiles && (wb >> 7) && w == 0)) { corrupt = true; w = 0; }
                words += w ? 1u + w : 0u;
            }
        }
        if (topo) {
#pragma unroll
            for (int j = 0; j < DT_BLOCKS * 2 / 32; j++)
                cps += __popc(label_word(labels, t * DT_BLOCKS * 2 + j * 32 + lane, g.n) & 0x55555555u);
        }
        words = __reduce_add_sync(FULL, words);
        cps = __reduce_add_sync(FULL, cps);
        if (lane == 0) {
            tile_w[t] = words;
            tile_c[t] = cps;
            unsigned long long* sl = s_sl[t / slice_len(ntiles)];
            if (words) atomicAdd(sl, (unsigned long long)words);
            if (cps) atomicAdd(sl + 1, (unsigned long long)cps);
        }
    }
    if (topo) {   // payload words of the rank stream's tiles (8192 deltas each)
        const uint8_t* rwidths = in + lo.r2;
        const uint32_t nbd = (uint32_t)cdiv(c->k_total, L);
        const uint32_t nrt = (nbd + DT_BLOCKS - 1) / DT_BLOCKS;
        for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nrt; t += (gridDim.x * blockDim.x) >> 5) {
            uint32_t words = 0;
#pragma unroll
            for (int j = 0; j < DT_BLOCKS / 32; j++) {
                const uint32_t b = t * DT_BLOCKS + j * 32 + lane;
                if (b < nbd) {
                    uint32_t w = __ldg(rwidths + b);
                    if (w > 32) { corrupt = true; w = 0; }
                    words += w ? 1u + w : 0u;
                }
            }
            words = __reduce_add_sync(FULL, words);
            if (lane == 0) {
                rtile_w[t] = words;
                if (words) atomicAdd(&s_sl[t / slice_len(nrt)][2], (unsigned long long)words);
            }
        }
    }
    if (corrupt) set_status(status, ST_CORRUPT);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < SCAN_SLICES * 3; i += blockDim.x) {
        const unsigned long long v = s_sl[i / 3][i % 3];
        if (v) atomicAdd(i % 3 < 2 ? &c->sl_tile[i / 3][i % 3] : &c->sl_rank[i / 3][0], v);
    }
}

// exclusive scans of the tile sums (slice-parallel: the sums of each slice
// were added up by k_dec_tile_sums); totals must match the header.
__global__ void __launch_bounds__(1024) k_dec_tile_scan(Ctrl* c, const uint32_t* tile_w, const uint32_t* tile_c,
                                                        unsigned long long* pay_pre, uint32_t* cp_pre,
                                                        uint32_t* rtile_w, int* status) {
    griddep_enter();
    __shared__ unsigned long long s_w[33][2];
    if (*status) return;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (!(c->flags & FLAG_NO_TOPO)) {   // the rank stream's tile prefixes, in place
        const uint32_t nbd = (uint32_t)cdiv(c->k_total, L);
        const uint32_t nrt = (nbd + DT_BLOCKS - 1) / DT_BLOCKS;
        unsigned long long rw, rz;
        slice_scan_pairs(
            nrt, c->sl_rank, [&](uint32_t i) { return make_uint2(rtile_w[i], 0u); },
            [&](uint32_t i, unsigned long long pw, unsigned long long) { rtile_w[i] = (uint32_t)pw; }, s_w, rw, rz);
        if (lead) {
            rtile_w[nrt] = (uint32_t)rw;
            if (rw != c->rank_words) set_status(status, ST_CORRUPT);
        }
    }
    const uint32_t ntiles = all_tiles(c->g);
    unsigned long long tw, tc;
    slice_scan_pairs(
        ntiles, c->sl_tile, [&](uint32_t i) { return make_uint2(tile_w[i], tile_c[i]); },
        [&](uint32_t i, unsigned long long pw, unsigned long long pc) {
            pay_pre[i] = pw;
            cp_pre[i] = (uint32_t)pc;
        },
        s_w, tw, tc);
    if (lead) {
        pay_pre[ntiles] = tw;
        cp_pre[ntiles] = (uint32_t)tc;
        const bool topo = !(c->flags & FLAG_NO_TOPO);
        if (tw != c->pay_words || (topo && tc != c->k_total)) set_status(status, ST_CORRUPT);
    }
}

// ------------------------------------------------------- fused wavefront decode
//
// One persistent kernel over linear tiles of 8192 points.  The CTA that takes
// tile t runs
//   S1(t)       decode: BE^, LZ^ + B^, QZ^ -> out = D0; positions of extrema
//   S2(t - H)   CP^ + RP^ evaluation of that tile's extrema on the D0 snapshot
//   S3(t - 2H)  apply the accepted stencil values
//   S4(t - 3H)  collect the tile's saddles that are still lost
// where H tiles cover the farthest face neighbour (one plane in 3D, one row in
// 2D).  Stage k of tile s starts only when stage k-1 is complete for every tile
// up to s + H (a per-stage frontier over per-tile flags), so S2 always reads
// unmodified D0 (Jacobi, as in the oracle) and S4 reads finished extrema, while
// the working window of about 3H tiles stays in L2: the field reaches HBM once.
// Waits only ever point at lower tile indices held by running CTAs (tiles are
// handed out in order), and every wait is bounded.

struct CgVal {   // L2-coherent reads of a field other CTAs write during the kernel
    const float* F;
    __device__ __forceinline__ float operator()(uint32_t j) const { return __ldcg(F + j); }
};

// Warp 0 waits until stage `k` is complete for every tile below `need`.  A
// wait also ends once the status word is set (polled every 64 fruitless
// polls): after one wait has run out, or a stage found a damaged stream, the
// others stop waiting for work that will not come.
__device__ __forceinline__ void wait_front(Ctrl* c, const uint32_t* flags, int k, uint32_t need,
                                           uint32_t ntiles, int* status) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        volatile unsigned int* fr = &c->front[k];
        uint32_t spins = 0;
        while (true) {
            // one read, broadcast: every branch below must be warp-uniform,
            // since the loop body uses full-warp ballots
            uint32_t f = 0;
            int stv = 0;
            if (lane == 0) {
                f = *fr;
                if ((spins & 63u) == 63u) stv = *(volatile int*)status;
            }
            f = __shfl_sync(FULL, f, 0);
            stv = __shfl_sync(FULL, stv, 0);
            if (f >= need || stv) break;
            const uint32_t j = f + lane;
            const uint32_t v = j < ntiles ? *(volatile const uint32_t*)(flags + j) : 0u;
            const uint32_t done = __ballot_sync(FULL, (v >> k) & 1u);
            const uint32_t run = done == FULL ? 32u : (uint32_t)(__ffs(~done) - 1);
            if (run) {
                if (lane == 0) atomicMax((unsigned int*)&c->front[k], f + run);
                continue;
            }
            if (++spins > SPIN_LIMIT) {
                if (lane == 0) set_status(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(spins < 64 ? 32 : 256);
        }
        __threadfence();
    }
    __syncthreads();
}

// Publish stage k of `tile` (waiters advance the frontier, 32 tiles per poll).
__device__ __forceinline__ void mark_done(Ctrl* c, uint32_t* flags, int k, uint32_t tile, uint32_t ntiles) {
    (void)c;
    (void)ntiles;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicOr(flags + tile, 1u << k);
    }
}

// Tiles between a point and its farthest face neighbour (+1 for the tile
// boundary, +1 spare), capped at the tile count.
__host__ __device__ inline uint32_t fused_reach(const Geo& g, uint32_t ntiles) {
    const uint32_t reach = g.ndim == 3 ? g.nxy : g.nx;
    const uint32_t h = reach / (DT_BLOCKS * L) + 2;
    return h < ntiles ? h : ntiles;
}

struct FusedArgs {
    const uint8_t* in;
    Ctrl* c;
    float* out;
    const unsigned long long* pay_pre;
    const uint32_t* cp_pre;
    const int32_t* delta;
    uint32_t* cp_idx;
    float* newv;
    uint32_t* flags;
    uint32_t* sad;
    uint32_t sad_cap;
    uint32_t slack;
    int* status;
};

// S1 for tile t, one block per thread: the tile's payload is staged in shared
// memory with coalesced loads; every thread finds its block's words from a
// CTA-wide scan of the widths, rebuilds the 32 magnitudes from the planes with
// register bit operations, applies the signs and the Lorenzo prefix, and
// writes D0 through a padded shared buffer so that the stores are coalesced.
// TOPO: the tile's extrema positions, in index order, go to cp_idx (bit 31:
// the point is a maximum).
constexpr int DT_ROW = 36;   // shared words per staged output row (conflict-free 16-byte accesses)

template <bool TOPO>
__device__ void stage_decode(const FusedArgs& A, const Geo& g, const Layout& lo, uint32_t t, uint32_t* s_pay,
                             uint32_t* s_w, uint32_t* s_cp, bool& corrupt) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t* widths = A.in + lo.s2;
    const int32_t* firsts = reinterpret_cast<const int32_t*>(A.in + lo.s4);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(A.in + lo.s5);
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(A.in + lo.s6);
    const float w_f = A.c->w_f;
    // this thread's block: width, first code, labels (issued before the payload
    // loads, so that both are in flight together)
    const uint32_t b = t * DT_BLOCKS + threadIdx.x;
    uint32_t w = 0, l0 = 0, l1 = 0;
    int32_t first = 0;
    if (b < g.nb) {
        w = __ldg(widths + b);
        first = __ldg(firsts + b);
        if (TOPO) {
            l0 = label_word(labels, 2 * b, g.n);
            l1 = label_word(labels, 2 * b + 1, g.n);
        }
    }
    // the tile's payload is one contiguous word range: stage it with coalesced loads
    const unsigned long long P0 = A.pay_pre[t], P1 = A.pay_pre[t + 1];
    uint32_t len = 0;
    if (P1 >= P0 && P1 - P0 <= (unsigned long long)DT_BLOCKS * 33 && P1 <= A.c->pay_words) len = (uint32_t)(P1 - P0);
    else corrupt = true;
    for (uint32_t i0 = 0; i0 < len; i0 += 4 * DT_BLOCKS) {   // four loads in flight per thread
        uint32_t v4[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t i = i0 + j * DT_BLOCKS + threadIdx.x;
            v4[j] = i < len ? __ldg(pay + P0 + i) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t i = i0 + j * DT_BLOCKS + threadIdx.x;
            if (i < len) s_pay[i] = v4[j];
        }
    }
    if (w > 32) w = 0;   // a damaged stream (the offset pre-pass flags it)
    uint32_t xm = 0, xM = 0;
    if (TOPO) {   // m = 01, M = 11: the low bit marks an extremum
        xm = compact16(l0) | compact16(l1) << 16;
        xM = compact16(l0 & (l0 >> 1)) | compact16(l1 & (l1 >> 1)) << 16;
    }
    const uint32_t words = w ? 1u + w : 0u, ncp = __popc(xm);
    uint32_t iw = words, ic = ncp;
#pragma unroll
    for (int of = 1; of < 32; of <<= 1) {
        const uint32_t a0 = __shfl_up_sync(FULL, iw, of), a1 = __shfl_up_sync(FULL, ic, of);
        if (lane >= (uint32_t)of) { iw += a0; ic += a1; }
    }
    if (lane == 31) {
        s_w[warp] = iw;
        s_cp[warp] = ic;
    }
    __syncthreads();
    uint32_t woff = iw - words, cpl = ic - ncp;
    for (uint32_t k = 0; k < warp; k++) {
        woff += s_w[k];
        cpl += s_cp[k];
    }
    // magnitudes from the planes (a transpose, see planes_to_values), then
    // signs and the Lorenzo prefix
    uint32_t v[32];
    uint32_t sgn = 0;
    uint32_t wv = w;   // planes present (0: constant block or a damaged stream)
    if (w && woff + 1 + w > len) {
        corrupt = true;
        wv = 0;
    }
    if (wv) sgn = s_pay[woff];
    planes_to_values(__reduce_max_sync(FULL, wv), wv, [&](int r) { return s_pay[woff + 1 + r]; }, v);
    {
        int32_t q = first;
#pragma unroll
        for (int e = 0; e < 32; e++) {
            if (e) q += (sgn >> e) & 1u ? -(int32_t)v[e] : (int32_t)v[e];
            v[e] = __float_as_uint(dequantize(q, w_f));
        }
    }
    __syncthreads();   // the payload is consumed: the buffer stages the output rows
    {
        uint32_t* row = s_pay + threadIdx.x * DT_ROW;
#pragma unroll
        for (int k = 0; k < 8; k++)
            *reinterpret_cast<uint4*>(row + 4 * k) = make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    if (TOPO && xm) {
        const unsigned long long k = A.c->k_total;
        unsigned long long pos = A.cp_pre[t] + cpl;
        while (xm) {
            const int e = __ffs(xm) - 1;
            xm &= xm - 1;
            // bit 31 carries the type (1: maximum), so the stencil stage needs no label load
            if (pos < k) A.cp_idx[pos] = (b * 32u + (uint32_t)e) | ((xM >> e) & 1u) << 31;
            else corrupt = true;
            pos++;
        }
    }
    __syncthreads();
    const uint64_t p0 = (uint64_t)t * (DT_BLOCKS * 32);
    const uint64_t left = (uint64_t)g.n - p0;
    if (left >= (uint64_t)(DT_BLOCKS * 32) && (reinterpret_cast<uintptr_t>(A.out) & 15u) == 0) {
        float4* dst = reinterpret_cast<float4*>(A.out + p0);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t idx = k * 256 + threadIdx.x;
            dst[idx] = *reinterpret_cast<const float4*>(s_pay + (idx >> 3) * DT_ROW + (idx & 7) * 4);
        }
    } else {
        const uint32_t np = left < (uint64_t)(DT_BLOCKS * 32) ? (uint32_t)left : (uint32_t)(DT_BLOCKS * 32);
        for (uint32_t i = threadIdx.x; i < np; i += blockDim.x)
            A.out[p0 + i] = __uint_as_float(s_pay[(i >> 5) * DT_ROW + (i & 31)]);
    }
}

// CP^ + RP^ on one tile's extrema, reading the D0 snapshot (Jacobi).  Each
// neighbour is loaded once and serves both the lost test and the extreme
// neighbour value.  Threads take two extrema at a time, all loads first.
struct ExtIn {
    float v0, u[6];
    long long dl;
    int lab;
    uint32_t have;   // bit e: neighbour e exists, (x-, x+, y-, y+, z-, z+)
    bool ok;
};

__device__ __forceinline__ void ext_load(const FusedArgs& A, const Geo& g, const uint32_t* labels, uint32_t pos,
                                         ExtIn& e) {
    const uint32_t raw = __ldcg(A.cp_idx + pos);
    const uint32_t p = raw & 0x7FFFFFFFu;
    e.ok = p < g.n;   // only a damaged stream fails this (its checks already failed)
    if (!e.ok) return;
    const uint32_t st[3] = {1u, g.nx, g.nxy};
    e.lab = raw >> 31 ? LAB_MAX : LAB_MIN;
    e.dl = __ldg(A.delta + pos);
    uint32_t x, y, z;
    coords(g, p, x, y, z);
    const uint32_t cc[3] = {x, y, z}, dd[3] = {g.nx, g.ny, g.nz};
    e.v0 = __ldcg(A.out + p);
    e.have = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        const bool on = ax < g.ndim;
        const bool lo = on && cc[ax] > 0, hi = on && cc[ax] + 1 < dd[ax];
        e.have |= (lo ? 1u : 0u) << (2 * ax) | (hi ? 1u : 0u) << (2 * ax + 1);
        e.u[2 * ax] = lo ? __ldcg(A.out + p - st[ax]) : 0.0f;
        e.u[2 * ax + 1] = hi ? __ldcg(A.out + p + st[ax]) : 0.0f;
    }
}

__device__ __forceinline__ float ext_eval(const ExtIn& e, float h_f, uint32_t& restored, uint32_t& skipped) {
    float nv = __int_as_float(0x7FC00000);
    if (!e.ok) return nv;
    // type of p in D0: for a labelled extremum only m / M matter (no FT)
    int nn = 0, nhi = 0, nlo = 0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        if (!((e.have >> k) & 1u)) continue;
        nn++;
        nhi += e.u[k] > e.v0;
        nlo += e.u[k] < e.v0;
    }
    const bool kept = nn > 0 && (e.lab == LAB_MIN ? nhi == nn : nlo == nn);
    if (!kept) {
        float ext = 0.0f;
        bool any = false;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            if (!((e.have >> k) & 1u)) continue;
            if (!any || (e.lab == LAB_MAX ? e.u[k] > ext : e.u[k] < ext)) ext = e.u[k];
            any = true;
        }
        float v;
        if (any && step_ulps(ext, e.lab == LAB_MAX ? e.dl : -e.dl, v) && fabsf(__fsub_rn(v, e.v0)) <= h_f) {
            nv = v;
            restored++;
        } else {
            skipped++;
        }
    }
    return nv;
}

// An interior extremum (all face neighbours present, nearly every one): p is
// kept iff the extreme neighbour value stays strictly on its side, and that
// value is the one stepped -- ext_eval's rule with every neighbour present,
// as one max (min) of the 4 or 6 neighbours.
__device__ __forceinline__ float ext_interior(const FusedArgs& A, const Geo& g, uint32_t p, bool is_max,
                                              long long dl, float h_f, uint32_t& restored, uint32_t& skipped) {
    const float v0 = __ldcg(A.out + p);
    const float u0 = __ldcg(A.out + p - 1), u1 = __ldcg(A.out + p + 1);
    const float u2 = __ldcg(A.out + p - g.nx), u3 = __ldcg(A.out + p + g.nx);
    float m = is_max ? fmaxf(fmaxf(u0, u1), fmaxf(u2, u3)) : fminf(fminf(u0, u1), fminf(u2, u3));
    if (g.ndim == 3) {
        const float u4 = __ldcg(A.out + p - g.nxy), u5 = __ldcg(A.out + p + g.nxy);
        m = is_max ? fmaxf(m, fmaxf(u4, u5)) : fminf(m, fminf(u4, u5));
    }
    if (is_max ? m < v0 : m > v0) return __int_as_float(0x7FC00000);   // kept
    float v;
    if (step_ulps(m, is_max ? dl : -dl, v) && fabsf(__fsub_rn(v, v0)) <= h_f) {
        restored++;
        return v;
    }
    skipped++;
    return __int_as_float(0x7FC00000);
}

__device__ void stage_extrema(const FusedArgs& A, const Geo& g, const uint32_t* labels, uint32_t s,
                              uint32_t& restored, uint32_t& skipped) {
    const uint32_t P0 = A.cp_pre[s], P1 = A.cp_pre[s + 1];
    const float h_f = A.c->h_f;
    for (uint32_t pos = P0 + threadIdx.x; pos < P1; pos += blockDim.x) {
        const uint32_t raw = __ldcg(A.cp_idx + pos);
        const uint32_t p = raw & 0x7FFFFFFFu;
        float nv = __int_as_float(0x7FC00000);
        if (p < g.n) {   // only a damaged stream fails this (its checks already failed)
            uint32_t x, y, z;
            coords(g, p, x, y, z);
            if (is_interior(g, x, y, z)) {
                nv = ext_interior(A, g, p, raw >> 31, __ldg(A.delta + pos), h_f, restored, skipped);
            } else {
                ExtIn e1;
                ext_load(A, g, labels, pos, e1);
                nv = ext_eval(e1, h_f, restored, skipped);
            }
        }
        A.newv[pos] = nv;
    }
}

__device__ void stage_apply(const FusedArgs& A, const Geo& g, uint32_t s) {
    const uint32_t P0 = A.cp_pre[s], P1 = A.cp_pre[s + 1];
    for (uint32_t pos = P0 + threadIdx.x; pos < P1; pos += blockDim.x) {
        const float v = __ldcg(A.newv + pos);
        const uint32_t p = __ldcg(A.cp_idx + pos) & 0x7FFFFFFFu;
        if (!isnan(v) && p < g.n) A.out[p] = v;
    }
}

// Saddles of tile s that the extrema stage left lost go to the candidate list.
// The tile's saddle labels are first compacted into shared memory, so that
// each thread then handles about one saddle with all of its loads in flight.
__device__ void stage_saddles(const FusedArgs& A, const Geo& g, const uint32_t* labels, uint32_t s,
                              uint32_t* s_list, uint32_t& s_cnt) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int part = 0; part < DT_BLOCKS * 2 / (int)blockDim.x; part++) {
        const uint32_t wi = s * DT_BLOCKS * 2 + part * blockDim.x + threadIdx.x;
        uint32_t smask = ((label_word(labels, wi, g.n) >> 1) & ~label_word(labels, wi, g.n)) & 0x55555555u;
        const uint32_t cnt = __popc(smask);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t tt = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += tt;
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        uint32_t base = 0;
        if (lane == 31 && tot) base = atomicAdd(&s_cnt, tot);
        uint32_t slot = __shfl_sync(FULL, base, 31) + incl - cnt;
        while (smask) {   // slots stay below the tile's point count
            const int bit = __ffs(smask) - 1;
            smask &= smask - 1;
            s_list[slot++] = wi * 16u + (uint32_t)(bit >> 1);
        }
    }
    __syncthreads();
    const uint32_t ns = s_cnt;
    CgVal val{A.out};
    const uint32_t st[3] = {1u, g.nx, g.nxy};
    const bool solve = A.c->flags & FLAG_RBF_SOLVE;   // no small-move filter: the step is unclamped
    for (uint32_t k0 = 0; k0 < ns; k0 += blockDim.x) {
        const uint32_t k = k0 + threadIdx.x;
        bool keep = false;
        if (k < ns) {
            const uint32_t p = s_list[k];
            uint32_t x, y, z;
            coords(g, p, x, y, z);
            if (!is_interior(g, x, y, z)) {
                keep = true;   // never a saddle off the interior: lost
            } else {
                const float fp = val(p);
                const int nd = g.ndim;
                float nb[6];
                bool nbsad = false;
#pragma unroll
                for (int ax = 0; ax < 3; ax++) {
                    if (ax >= nd) break;
                    nb[2 * ax] = val(p - st[ax]);
                    nb[2 * ax + 1] = val(p + st[ax]);
                    nbsad |= label_at(labels, p - st[ax]) == LAB_SAD || label_at(labels, p + st[ax]) == LAB_SAD;
                }
                int ph = 0, pl = 0, px = 0;
#pragma unroll
                for (int ax = 0; ax < 3; ax++) {
                    if (ax >= nd) break;
                    const float a = nb[2 * ax], b = nb[2 * ax + 1];
                    if (a > fp && b > fp) ph++;
                    else if (a < fp && b < fp) pl++;
                    else px++;
                }
                const bool lost = !(px == 0 && ph > 0 && pl > 0);
                // A lost saddle whose face neighbours never change during the
                // rounds (none of them is saddle-labelled) keeps its status for
                // good: if no small move of p can make it a saddle now, every
                // colour round would reject it, so it is not listed.
                keep = lost && (nbsad || solve || saddle_feasible(nb, nd, fp));
            }
        }
        const uint32_t bal = __ballot_sync(FULL, keep);
        uint32_t base = 0;
        if (lane == 0 && bal) base = atomicAdd(&A.c->sad_cnt[0], (unsigned)__popc(bal));
        base = __shfl_sync(FULL, base, 0);
        if (keep) {
            const uint32_t slot = base + __popc(bal & lanemask_lt());
            if (slot < A.sad_cap) A.sad[slot] = s_list[k];
        }
    }
}

struct FusedSmem {
    __align__(16) uint32_t pay[DT_BLOCKS * DT_ROW];   // S1: the tile's payload, then its output rows; S4: its saddle list
    uint32_t tile, cnt, hold;   // hold: the test hook's tile + 1 (0: none)
    Geo g;
    Layout lo;
    uint32_t w[DT_WARPS], cp[DT_WARPS];
};

template <bool TOPO>
__device__ void fused_body(const FusedArgs& A, FusedSmem& S) {
    uint32_t* s_pay = S.pay;
    uint32_t& s_tile = S.tile;
    uint32_t* s_w = S.w;
    uint32_t* s_cp = S.cp;
    Ctrl* c = A.c;
    // geometry and layout live in shared memory: read where used, not held in
    // registers across the stages
    if (threadIdx.x == 0) {
        S.g = c->g;
        S.lo = c->lo;
        S.hold = c->test_hold;
    }
    __syncthreads();
    const Geo& g = S.g;
    const Layout& lo = S.lo;
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(A.in + lo.s6);
    const uint32_t ntiles = lin_tiles(g);
    // format v2: S1 ran before (k_decode_tiles); S2 starts on a finished field
    const bool s1 = !(c->flags & FLAG_TILE_BLOCKS);
    const uint32_t H = TOPO ? fused_reach(g, ntiles) : 0u;
    // stage lag: the reach H plus some slack, so that a stage rarely waits for
    // tiles that CTAs took just before this one
    const uint32_t Lg = TOPO ? hmin<uint32_t>(H + A.slack, ntiles) : 0u;
    const uint32_t total = ntiles + 3 * Lg;
    bool corrupt = false;
    uint32_t restored = 0, skipped = 0;   // per thread: at most the extrema it handled
    while (true) {
    // a set status word ends the call: take no more tiles
    if (threadIdx.x == 0) s_tile = *(volatile int*)A.status ? total : atomicAdd(&c->tile_fused, 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    __syncthreads();
    if (t >= total) break;
    if (s1 && t < ntiles) {
        stage_decode<TOPO>(A, g, lo, t, s_pay, s_w, s_cp, corrupt);
        if (t + 1 != S.hold) mark_done(c, A.flags, 1, t, ntiles);
        else __syncthreads();   // the test hook: this tile is never published
    }
    if (TOPO) {
        const long long s2 = (long long)t - Lg, s3 = (long long)t - 2 * Lg, s4 = (long long)t - 3 * Lg;
        if (s2 >= 0 && s2 < ntiles) {
            if (s1) wait_front(c, A.flags, 1, (uint32_t)hmin<long long>(s2 + H, ntiles - 1) + 1, ntiles, A.status);
            stage_extrema(A, g, labels, (uint32_t)s2, restored, skipped);
            mark_done(c, A.flags, 2, (uint32_t)s2, ntiles);
        }
        if (s3 >= 0 && s3 < ntiles) {
            wait_front(c, A.flags, 2, (uint32_t)hmin<long long>(s3 + H, ntiles - 1) + 1, ntiles, A.status);
            stage_apply(A, g, (uint32_t)s3);
            mark_done(c, A.flags, 3, (uint32_t)s3, ntiles);
        }
        if (s4 >= 0 && s4 < ntiles) {
            wait_front(c, A.flags, 3, (uint32_t)hmin<long long>(s4 + H, ntiles - 1) + 1, ntiles, A.status);
            stage_saddles(A, g, labels, (uint32_t)s4, s_pay, S.cnt);
        }
    }
    }
    if (corrupt) set_status(A.status, ST_CORRUPT);
    if (TOPO) {
        for (int o = 16; o > 0; o >>= 1) {
            restored += __shfl_xor_sync(FULL, restored, o);
            skipped += __shfl_xor_sync(FULL, skipped, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (restored) atomicAdd(&c->stat_restored, (unsigned long long)restored);
            if (skipped) atomicAdd(&c->stat_skipped, (unsigned long long)skipped);
        }
    }
}

__global__ void __launch_bounds__(256, 4) k_decode_fused(FusedArgs A) {
    griddep_enter();
    __shared__ FusedSmem S;
    if (*A.status) return;
    if (A.c->flags & FLAG_NO_TOPO) fused_body<false>(A, S);
    else fused_body<true>(A, S);
}

// The same four stages as separate launches (one CTA per tile per stage; the
// kernel boundaries order the stages, so there are no waits).
template <int K>
__global__ void __launch_bounds__(256, 4) k_decode_stage(FusedArgs A) {
    griddep_enter();
    __shared__ FusedSmem S;
    if (*A.status) return;
    Ctrl* c = A.c;
    const bool topo = !(c->flags & FLAG_NO_TOPO);
    if (K > 1 && !topo) return;
    if (K == 1 && (c->flags & FLAG_TILE_BLOCKS)) return;   // format v2: k_decode_tiles is S1
    if (threadIdx.x == 0) {
        S.g = c->g;
        S.lo = c->lo;
    }
    __syncthreads();
    const Geo& g = S.g;
    const Layout& lo = S.lo;
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(A.in + lo.s6);
    const uint32_t ntiles = lin_tiles(g);
    bool corrupt = false;
    uint32_t restored = 0, skipped = 0;   // per thread: at most the extrema it handled
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (K == 1) {
            if (topo) stage_decode<true>(A, g, lo, t, S.pay, S.w, S.cp, corrupt);
            else stage_decode<false>(A, g, lo, t, S.pay, S.w, S.cp, corrupt);
            __syncthreads();
        } else if (K == 2) {
            stage_extrema(A, g, labels, t, restored, skipped);
        } else if (K == 3) {
            stage_apply(A, g, t);
        } else {
            stage_saddles(A, g, labels, t, S.pay, S.cnt);
            __syncthreads();
        }
    }
    if (corrupt) set_status(A.status, ST_CORRUPT);
    if (K == 2) {
        for (int o = 16; o > 0; o >>= 1) {
            restored += __shfl_xor_sync(FULL, restored, o);
            skipped += __shfl_xor_sync(FULL, skipped, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (restored) atomicAdd(&c->stat_restored, (unsigned long long)restored);
            if (skipped) atomicAdd(&c->stat_skipped, (unsigned long long)skipped);
        }
    }
}

// ------------------------------------------------------- format v2: S1
//
// S1 for tile-shaped blocks (the inverse of k_encode_tiles): one payload tile
// of 256 blocks per CTA and step, one block per thread.  The tile's payload
// is staged in shared memory as in stage_decode; a thread rebuilds its
// block's residuals from the planes, undoes the coded predictor in 32-bit
// modular arithmetic (the chain: a prefix sum in element order; Lorenzo:
// prefix sums along x, then y, then z), adds q_0, dequantises and writes the
// points of the block that lie inside the grid.  For each linear tile the
// extremum positions go to cp_idx as S1 of format v1 writes them.  A
// format-v1 stream returns at once (the fused decoder's S1 decodes it).
template <int ND>
__device__ void tiles_decode_one(const uint8_t* in, const Ctrl* c, const Geo& g, const Layout& lo, float* out,
                                 const unsigned long long* pay_pre, uint32_t t, uint32_t* s_pay, uint32_t* s_w,
                                 bool& corrupt) {
    using TS = TileShape<ND>;
    constexpr uint32_t BX = TS::BX, BY = TS::BY, BZ = TS::BZ;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t* widths = in + lo.s2;
    const int32_t* firsts = reinterpret_cast<const int32_t*>(in + lo.s4);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(in + lo.s5);
    const uint32_t b = t * DT_BLOCKS + threadIdx.x;
    uint32_t wb = 0;
    int32_t first = 0;
    if (b < g.nb) {
        wb = __ldg(widths + b);
        first = __ldg(firsts + b);
    }
    const unsigned long long P0 = pay_pre[t], P1 = pay_pre[t + 1];
    uint32_t len = 0;
    if (P1 >= P0 && P1 - P0 <= (unsigned long long)DT_BLOCKS * 33 && P1 <= c->pay_words) len = (uint32_t)(P1 - P0);
    else corrupt = true;
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s_pay[i] = __ldg(pay + P0 + i);
    uint32_t w = wb & 0x7Fu, sel = wb >> 7;
    if (w > 32 || (sel && w == 0)) w = 0, sel = 0;   // a damaged stream (the tile sums flag it)
    const uint32_t words = w ? 1u + w : 0u;
    uint32_t iw = words;
#pragma unroll
    for (int of = 1; of < 32; of <<= 1) {
        const uint32_t a0 = __shfl_up_sync(FULL, iw, of);
        if (lane >= (uint32_t)of) iw += a0;
    }
    if (lane == 31) s_w[warp] = iw;
    __syncthreads();
    uint32_t woff = iw - words;
    for (uint32_t k = 0; k < warp; k++) woff += s_w[k];
    uint32_t wv = w;
    if (w && woff + 1 + w > len) {
        corrupt = true;
        wv = 0;
    }
    uint32_t v[32];
    const uint32_t sgn = wv ? s_pay[woff] : 0u;
    planes_to_values(__reduce_max_sync(FULL, wv), wv, [&](int r) { return s_pay[woff + 1 + r]; }, v);
#pragma unroll
    for (int e = 0; e < 32; e++) v[e] = (sgn >> e) & 1u ? 0u - v[e] : v[e];
    if (sel) {
#pragma unroll
        for (int e = 0; e < 32; e++)
            if ((uint32_t)e % BX) v[e] += v[e - 1];
#pragma unroll
        for (int e = 0; e < 32; e++)
            if (((uint32_t)e / BX) % BY) v[e] += v[e - BX];
#pragma unroll
        for (int e = 0; e < 32; e++)
            if ((uint32_t)e / (BX * BY)) v[e] += v[e - BX * BY];
    } else {
#pragma unroll
        for (int e = 1; e < 32; e++) v[e] += v[e - 1];
    }
    if (b < g.nb) {
        const float w_f = c->w_f;
        const uint32_t nbx = (g.nx + BX - 1) / BX, nby = (g.ny + BY - 1) / BY;
        const uint32_t gx = b % nbx, gy = (b / nbx) % nby, gz = b / (nbx * nby);
#pragma unroll
        for (int e = 0; e < 32; e++) {
            const uint32_t x = gx * BX + (uint32_t)e % BX, y = gy * BY + ((uint32_t)e / BX) % BY,
                           z = gz * BZ + (uint32_t)e / (BX * BY);
            if (x < g.nx && y < g.ny && z < g.nz)
                out[(size_t)x + (size_t)g.nx * (y + (size_t)g.ny * z)] =
                    dequantize((int32_t)(v[e] + (uint32_t)first), w_f);
        }
    }
    __syncthreads();   // s_pay and s_w are reused by the next step
}

// the extremum positions of linear tile t, in index order (bit 31: a maximum)
__device__ void tiles_cp_list(const uint8_t* in, const Ctrl* c, const Geo& g, const Layout& lo,
                              const uint32_t* cp_pre, uint32_t* cp_idx, uint32_t t, uint32_t* s_cp, bool& corrupt) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(in + lo.s6);
    const uint32_t bl = t * DT_BLOCKS + threadIdx.x;   // a linear block of 32 points: two label words
    const uint32_t l0 = label_word(labels, 2 * bl, g.n), l1 = label_word(labels, 2 * bl + 1, g.n);
    uint32_t xm = compact16(l0) | compact16(l1) << 16;
    const uint32_t xM = compact16(l0 & (l0 >> 1)) | compact16(l1 & (l1 >> 1)) << 16;
    const uint32_t ncp = __popc(xm);
    uint32_t ic = ncp;
#pragma unroll
    for (int of = 1; of < 32; of <<= 1) {
        const uint32_t a1 = __shfl_up_sync(FULL, ic, of);
        if (lane >= (uint32_t)of) ic += a1;
    }
    if (lane == 31) s_cp[warp] = ic;
    __syncthreads();
    uint32_t cpl = ic - ncp;
    for (uint32_t k = 0; k < warp; k++) cpl += s_cp[k];
    const unsigned long long k = c->k_total;
    unsigned long long pos = cp_pre[t] + cpl;
    while (xm) {
        const int e = __ffs(xm) - 1;
        xm &= xm - 1;
        if (pos < k) cp_idx[pos] = (bl * 32u + (uint32_t)e) | ((xM >> e) & 1u) << 31;
        else corrupt = true;
        pos++;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_decode_tiles(const uint8_t* __restrict__ in, Ctrl* c, float* out,
                                                      const unsigned long long* pay_pre, const uint32_t* cp_pre,
                                                      uint32_t* cp_idx, int* status) {
    griddep_enter();
    __shared__ __align__(16) uint32_t s_pay[DT_BLOCKS * 33];
    __shared__ uint32_t s_w[DT_WARPS], s_cp[DT_WARPS];
    if (*status || !(c->flags & FLAG_TILE_BLOCKS)) return;
    const Geo g = c->g;
    const Layout lo = c->lo;
    const bool topo = !(c->flags & FLAG_NO_TOPO);
    const uint32_t npt = (g.nb + DT_BLOCKS - 1) / DT_BLOCKS, nlt = lin_tiles(g), nt = hmax(npt, nlt);
    bool corrupt = false;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {   // uniform across the CTA
        if (t < npt) {
            if (g.ndim == 3) tiles_decode_one<3>(in, c, g, lo, out, pay_pre, t, s_pay, s_w, corrupt);
            else tiles_decode_one<2>(in, c, g, lo, out, pay_pre, t, s_pay, s_w, corrupt);
        }
        if (topo && t < nlt) tiles_cp_list(in, c, g, lo, cp_pre, cp_idx, t, s_cp, corrupt);
    }
    if (corrupt) set_status(status, ST_CORRUPT);
}

// RS^ colour rounds over the lost-saddle list (cooperative: the grid syncs
// between the evaluation and the write of every colour).  The list is first
// bucketed by colour so that each round touches only its own candidates.
__global__ void __launch_bounds__(1024, 1) k_saddle_rounds(const uint8_t* __restrict__ in, Ctrl* c, float* out,
                                                       const uint32_t* sad, uint32_t* sadb, float* sadv,
                                                       uint32_t sad_cap, uint32_t* rec, uint32_t rec_cap,
                                                       int* status) {
    // a cooperative launch, without programmatic serialisation: it starts
    // after the previous kernel has completed, so it needs no griddep_enter()
    __shared__ RbfTable T;
    __shared__ uint32_t s_cnt[8], s_base[8];
    cg::grid_group grid = cg::this_grid();
    // uniform across the grid: neither word is written by this kernel
    if (*status || (c->flags & FLAG_NO_TOPO)) return;
    const Geo g = c->g;
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(in + c->lo.s6);
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const uint32_t ns = hmin<uint32_t>(c->sad_cnt[0], sad_cap);
    const int ncol = g.ndim == 2 ? 5 : 7;
    build_rbf_table(T, g, c);
    // bucket by colour
    if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t j = tid; j < ns; j += nth) {
        uint32_t x, y, z;
        coords(g, sad[j], x, y, z);
        atomicAdd(&s_cnt[colour_of(g, x, y, z)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 8 && s_cnt[threadIdx.x]) atomicAdd(&c->sad_col[threadIdx.x], s_cnt[threadIdx.x]);
    grid.sync();
    uint32_t base[8], cnt[8];
    {
        uint32_t b = 0;
        for (int k = 0; k < 8; k++) {
            base[k] = b;
            cnt[k] = *(volatile unsigned int*)&c->sad_col[k];
            b += cnt[k];
        }
    }
    // each block reserves one range per colour, then fills it through shared memory
    if (threadIdx.x < 8) {
        s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&c->sad_fill[threadIdx.x], s_cnt[threadIdx.x]) : 0u;
        s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    // records (uniform across the grid): when the kind has them and they fit
    const int r = c->rbf_k / 2;
    const bool use_rec = rec_cap > 0 && ns <= rec_cap && rec_supported(g.ndim, r);
    const uint32_t RW = use_rec ? rec_words(g.ndim, r) : REC_MAX_WORDS;   // rec_cap counts REC_MAX_WORDS each
    for (uint32_t j = tid; j < ns; j += nth) {
        const uint32_t p = sad[j];
        uint32_t x, y, z;
        coords(g, p, x, y, z);
        const int col = colour_of(g, x, y, z);
        const uint32_t slot = base[col] + s_base[col] + atomicAdd(&s_cnt[col], 1u);
        sadb[slot] = p;
        if (use_rec)
            rec_gather_any(g.ndim, r, out, labels, g, p, x, y, z, rec_inside(g, r, x, y, z), rec + (size_t)slot * RW);
    }
    grid.sync();
    unsigned long long fixed = 0;
    for (int sw = 0; sw < c->rs_sweeps; sw++) {
        for (int col = 0; col < ncol; col++) {
            const uint32_t b0 = base[col], nc = cnt[col];
            // warps take 32 candidates at a time: evaluation costs vary a lot
            while (true) {
                uint32_t k0 = 0;
                if ((threadIdx.x & 31) == 0) k0 = atomicAdd(&c->sad_next[col], 32u);
                k0 = __shfl_sync(FULL, k0, 0);
                if (k0 >= nc) break;
                const uint32_t j = k0 + (threadIdx.x & 31);
                if (j < nc) {
                    const uint32_t p = sadb[b0 + j];
                    float v;
                    bool ok;
                    if (use_rec) {
                        ok = saddle_candidate_rec_any(g.ndim, r, out, labels, g, c, T.den_full, p,
                                                      rec + (size_t)(b0 + j) * RW, v);
                    } else {
                        uint32_t x, y, z;
                        coords(g, p, x, y, z);
                        ok = saddle_candidate(out, labels, g, c, T, p, x, y, z, v);
                    }
                    sadv[b0 + j] = ok ? v : __int_as_float(0x7FC00000);
                }
            }
            grid.sync();
            // the counter is next used a sweep later, many grid syncs away
            if (tid == 0) c->sad_next[col] = 0;
            for (uint32_t j = tid; j < nc; j += nth) {
                const float v = sadv[b0 + j];
                if (!isnan(v)) {
                    out[sadb[b0 + j]] = v;
                    fixed++;
                }
            }
            grid.sync();
        }
    }
    for (int o = 16; o > 0; o >>= 1) fixed += __shfl_xor_sync(FULL, fixed, o);
    if ((threadIdx.x & 31) == 0 && fixed) atomicAdd(&c->stat_saddle, fixed);
}
// ------------------------------------------------------------ host launchers

void launch_parse_header(const uint8_t* in, uint64_t in_size, uint64_t n_out, Ctrl* c, int* status,
                         uint32_t test_hold, cudaStream_t st) {
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(k_parse_header, cudaFuncAttributeMaxDynamicSharedMemorySize, RBF_SOLVE_SMEM);
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    launch_pdl(k_parse_header, dim3(1), dim3(256), RBF_SOLVE_SMEM, st, in, in_size, n_out, c, status, test_hold);
}

void launch_decode_tiles(const uint8_t* in, Ctrl* c, float* out, const unsigned long long* pay_pre,
                         const uint32_t* cp_pre, uint32_t* cp_idx, uint64_t n, int sms, int* status,
                         cudaStream_t st) {
    // a format-v2 stream has at most n blocks; the CTAs step over the tiles
    const uint32_t grid = (uint32_t)hmax<uint64_t>(1, hmin<uint64_t>(cdiv(n, DT_BLOCKS), (uint64_t)sms * 8));
    launch_pdl(k_decode_tiles, dim3(grid), dim3(256), 0, st, in, c, out, pay_pre, cp_pre, cp_idx, status);
}

void launch_decode_ranks(const uint8_t* in, Ctrl* c, const uint32_t* rpre, int32_t* delta, uint64_t max_k,
                         int sms, int* status, cudaStream_t st) {
    uint32_t grid = hmin<uint32_t>((uint32_t)cdiv(cdiv(max_k, L), DT_BLOCKS), (uint32_t)sms * 3);
    if (grid == 0) grid = 1;
    launch_pdl(k_decode_ranks, dim3(grid), dim3(256), 0, st, in, c, rpre, delta, status);
}

void launch_dec_offsets(const uint8_t* in, Ctrl* c, uint32_t* tile_w, uint32_t* tile_c,
                        unsigned long long* pay_pre, uint32_t* cp_pre, uint32_t* rtile_w, uint32_t ntiles, int sms,
                        int* status, cudaStream_t st) {
    uint32_t blocks = hmin<uint32_t>((ntiles + 7) / 8, (uint32_t)sms * 8);
    if (blocks == 0) blocks = 1;
    launch_pdl(k_dec_tile_sums, dim3(blocks), dim3(256), 0, st, in, c, tile_w, tile_c, rtile_w, status);
    launch_pdl(k_dec_tile_scan, dim3(SCAN_SLICES), dim3(1024), 0, st, c, tile_w, tile_c, pay_pre, cp_pre, rtile_w, status);
}

void launch_decode_fused(const uint8_t* in, Ctrl* c, float* out, const unsigned long long* pay_pre,
                         const uint32_t* cp_pre, const int32_t* delta, uint32_t* cp_idx, float* newv,
                         uint32_t* flags, uint32_t* sad, uint32_t sad_cap, uint32_t ntiles_dec, uint32_t h_bound,
                         int sms, int* status, cudaStream_t st) {
    static int fit = -1;
    if (fit < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_decode_fused, 256, 0) != cudaSuccess || b < 1) b = 1;
        fit = b;
    }
    const uint32_t slack = g_tuning.dec_slack_tiles > 0 ? (uint32_t)g_tuning.dec_slack_tiles
                                                        : (uint32_t)(fit * sms) / 4u;
    FusedArgs A{in, c, out, pay_pre, cp_pre, delta, cp_idx, newv, flags, sad, sad_cap, slack, status};
    // About one virtual tile per CTA (ntiles decode tiles plus 3H trailing stage
    // slots; H is known only on the device, so CTAs keep taking virtual tiles
    // until all are done).  Waits only point at lower tiles, taken by CTAs that
    // started earlier, so any residency makes progress.
    if (g_tuning.dec_split > 0) {
        const uint32_t sg = hmin<uint32_t>(ntiles_dec, (uint32_t)(fit * sms) * 4u);
        launch_pdl(k_decode_stage<1>, dim3(sg), dim3(256), 0, st, A);
        launch_pdl(k_decode_stage<2>, dim3(sg), dim3(256), 0, st, A);
        launch_pdl(k_decode_stage<3>, dim3(sg), dim3(256), 0, st, A);
        launch_pdl(k_decode_stage<4>, dim3(sg), dim3(256), 0, st, A);
        return;
    }
    const uint32_t grid = ntiles_dec + 3 * hmin<uint32_t>(ntiles_dec, h_bound + slack);
    launch_pdl(k_decode_fused, dim3(grid), dim3(256), 0, st, A);
}

cudaError_t launch_saddle_rounds(const uint8_t* in, Ctrl* c, float* out, const uint32_t* sad, uint32_t* sadb,
                                 float* sadv, uint32_t sad_cap, uint32_t* rec, uint64_t rec_bytes, int sms,
                                 int* status, cudaStream_t st) {
    // 1024 threads per SM, as one CTA by default (the grid syncs are cheaper
    // with fewer CTAs) or split into 2 or 4
    const int per_sm = g_tuning.rounds_blocks_per_sm > 0 ? g_tuning.rounds_blocks_per_sm : 1;
    const int th = 1024 / per_sm;
    static int fit[5] = {-1, -1, -1, -1, -1};
    if (fit[per_sm] < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_saddle_rounds, th, 0) != cudaSuccess) b = 0;
        fit[per_sm] = b;
    }
    if (fit[per_sm] < per_sm) return cudaErrorCooperativeLaunchTooLarge;   // the grid must be co-resident
    uint32_t rec_cap = 0;
    if (g_tuning.saddle_records >= 0)
        rec_cap = (uint32_t)hmin<uint64_t>(rec_bytes / (4ull * REC_MAX_WORDS), 0xFFFFFFFFull);
    void* args[] = {(void*)&in, (void*)&c, (void*)&out, (void*)&sad, (void*)&sadb, (void*)&sadv,
                    (void*)&sad_cap, (void*)&rec, (void*)&rec_cap, (void*)&status};
    return cudaLaunchCooperativeKernel((const void*)k_saddle_rounds, dim3(per_sm * sms), dim3(th), args, 0, st);
}
}  // namespace tsz
