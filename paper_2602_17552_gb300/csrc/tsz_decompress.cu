// tsz_decompress.cu -- decompression kernels (Section IV-B of arXiv 2602.17552).
//
//   k_parse_header   one thread: validate the stream header against the call
//                    and the buffer size, fill the control block
//   k_decode_field   BE^, LZ^ + B^, QZ^: unpack sign/magnitude planes with warp
//                    shuffles, inverse Lorenzo by a warp prefix sum, dequantise;
//                    a look-back over (payload words, extremum count) gives each
//                    tile its payload offset and each extremum its position in
//                    the delta sequence (MD^)
//   k_decode_ranks   the same inverse codec on the rank stream
//   k_fixup          cooperative kernel: CP^ + RP^ extrema stencils (evaluate
//                    on the QZ^ snapshot, then apply), collect lost saddles,
//                    then RS^ colour rounds (evaluate, grid sync, apply)
// Every read of the stream is bounds-checked against the validated header; a
// violation sets CORRUPT_STREAM and skips the access.
#include <cooperative_groups.h>

#include "tsz_internal.h"

namespace cg = cooperative_groups;

namespace tsz {

template <class T>
__device__ __forceinline__ T get(const uint8_t* h, int off) {
    return *reinterpret_cast<const T*>(h + off);
}

__global__ void k_parse_header(const uint8_t* in, uint64_t in_size, uint64_t n_out, Ctrl* c,
                               int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (in_size < HDR || get<uint32_t>(in, 0) != MAGIC || get<uint32_t>(in, 4) != VERSION ||
        get<uint32_t>(in, 12) != L) {
        set_status(status, ST_CORRUPT);
        return;
    }
    const int ndim = (int)get<uint32_t>(in, 8);
    const uint64_t nx = get<uint64_t>(in, 16), ny = get<uint64_t>(in, 24), nz = get<uint64_t>(in, 32);
    const uint32_t flags = get<uint32_t>(in, 40);
    bool ok = (ndim == 2 || ndim == 3) && nx >= 1 && ny >= 1 && nz >= 1 && nx < (1ull << 31) &&
              ny < (1ull << 31) && nz < (1ull << 31) && (ndim == 3 || nz == 1) && flags <= 1;
    const uint64_t n = ok ? nx * ny : 0;
    ok = ok && n < (1ull << 31) && n * nz < (1ull << 31) && n * nz == n_out &&
         get<uint64_t>(in, 104) == n_out && get<uint64_t>(in, 112) == cdiv(n_out, L);
    const float w_f = get<float>(in, 64), h_f = get<float>(in, 72);
    const int32_t rk = (int32_t)get<uint32_t>(in, 88);
    const uint32_t sweeps = get<uint32_t>(in, 96);
    const uint64_t kmin = get<uint64_t>(in, 120), kmax = get<uint64_t>(in, 128);
    const uint64_t pay = get<uint64_t>(in, 208), rpay = get<uint32_t>(in, 216);
    const bool topo = !(flags & FLAG_NO_TOPO);
    ok = ok && isfinite(w_f) && w_f > 0.0f && isfinite(h_f) && h_f >= 0.0f;
    ok = ok && (rk == 3 || rk == 5 || rk == 7) && sweeps >= 1 && sweeps <= 16;
    ok = ok && kmin <= cdiv(n_out, 2) && kmax <= cdiv(n_out, 2) && (topo || (kmin == 0 && kmax == 0));
    const uint64_t nb = cdiv(n_out, L);
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
    c->g = g;
    c->flags = flags;
    c->w_f = w_f;
    c->h_f = h_f;
    c->rbf_k = rk;
    c->rs_sweeps = (int)sweeps;
    c->pay_words = pay;
    c->rank_words = rpay;
    c->k_total = kmin + kmax;
    c->lo = lo;
    for (int i = 0; i < 9; i++) c->g_rbf[i] = get<float>(in, 220 + 4 * i);
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

template <bool TOPO>
__device__ __forceinline__ void decode_field_body(const uint8_t* __restrict__ in, Ctrl* c, Desc* desc,
                                                  float* __restrict__ out, uint32_t* cp_idx, int* status) {
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_w[TILE_WARPS], s_cp[TILE_WARPS];
    __shared__ unsigned long long s_pre_w, s_pre_cp;
    const Geo g = c->g;
    const Layout lo = c->lo;
    const float w_f = c->w_f;
    const unsigned long long pay_words = c->pay_words, k = c->k_total;
    const uint8_t* widths = in + lo.s2;
    const int32_t* firsts = reinterpret_cast<const int32_t*>(in + lo.s4);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(in + lo.s5);
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(in + lo.s6);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ntiles = (g.nb + TILE_BLOCKS - 1) / TILE_BLOCKS;
    const uint32_t lt = lanemask_lt();
    bool corrupt = false;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&c->tile_dec, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t blk0 = tile * TILE_BLOCKS + warp * BPW;
        uint32_t my_w = 0;
        int32_t my_first = 0;
        if (lane < BPW && blk0 + lane < g.nb) {
            my_w = widths[blk0 + lane];
            my_first = firsts[blk0 + lane];
            if (my_w > 32) {
                corrupt = true;
                my_w = 0;
            }
        }
        uint32_t ww = (lane < BPW && my_w) ? 1u + my_w : 0u;
        ww = __reduce_add_sync(FULL, ww);
        uint32_t mmask[BPW];
        uint32_t wcp = 0;
#pragma unroll
        for (int j = 0; j < BPW; j++) {
            mmask[j] = 0;
            if (TOPO) {
                const uint32_t b = blk0 + j;
                if (b < g.nb) {
                    const uint32_t i = b * 32u + lane;
                    const int lab = i < g.n ? label_at(labels, i) : 0;
                    mmask[j] = __ballot_sync(FULL, lab & 1);   // m = 01, M = 11
                    wcp += __popc(mmask[j]);
                }
            }
        }
        if (lane == 0) {
            s_w[warp] = ww;
            s_cp[warp] = wcp;
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t vw = lane < TILE_WARPS ? s_w[lane] : 0, vc = lane < TILE_WARPS ? s_cp[lane] : 0;
            uint32_t iw = vw, ic = vc;
#pragma unroll
            for (int o = 1; o < TILE_WARPS; o <<= 1) {
                uint32_t t0 = __shfl_up_sync(FULL, iw, o), t1 = __shfl_up_sync(FULL, ic, o);
                if (lane >= o) { iw += t0; ic += t1; }
            }
            uint32_t tw = __shfl_sync(FULL, iw, TILE_WARPS - 1), tc = __shfl_sync(FULL, ic, TILE_WARPS - 1);
            unsigned long long pw, pc;
            lookback(desc, tile, tw, tc, pw, pc, status);
            if (lane < TILE_WARPS) {
                s_w[lane] = iw - vw;
                s_cp[lane] = ic - vc;
            }
            if (lane == 0) {
                s_pre_w = pw;
                s_pre_cp = pc;
                if (tile == ntiles - 1 && (pw + tw != pay_words || (TOPO && pc + tc != k)))
                    set_status(status, ST_CORRUPT);
            }
        }
        __syncthreads();
        unsigned long long woff = s_pre_w + s_w[warp];
        unsigned long long cpoff = s_pre_cp + s_cp[warp];
#pragma unroll
        for (int j = 0; j < BPW; j++) {
            const uint32_t b = blk0 + j;
            if (b >= g.nb) break;
            const uint32_t w = __shfl_sync(FULL, my_w, j);
            const int32_t first = __shfl_sync(FULL, my_first, j);
            int32_t q = first;
            if (w) {
                if (woff + 1 + w <= pay_words) q = decode_block(pay, woff, w, first, lane);
                else corrupt = true;
                woff += 1 + w;
            }
            const uint32_t i = b * 32u + lane;
            if (i < g.n) out[i] = dequantize(q, w_f);
            if (TOPO) {
                const uint32_t mm = mmask[j];
                if ((mm >> lane) & 1u) {
                    unsigned long long pos = cpoff + __popc(mm & lt);
                    if (pos < k) cp_idx[pos] = i;
                    else corrupt = true;
                }
                cpoff += __popc(mm);
            }
        }
        __syncthreads();
    }
    if (corrupt) set_status(status, ST_CORRUPT);
}

// The stream's flags decide at run time whether labels are read (the host does
// not read the header, so one launch serves both kinds of stream).
__global__ void __launch_bounds__(256) k_decode_field(const uint8_t* __restrict__ in, Ctrl* c, Desc* desc,
                                                      float* __restrict__ out, uint32_t* cp_idx,
                                                      int* status) {
    if (*status) return;
    if (c->flags & FLAG_NO_TOPO) decode_field_body<false>(in, c, desc, out, cp_idx, status);
    else decode_field_body<true>(in, c, desc, out, cp_idx, status);
}

__global__ void __launch_bounds__(256) k_decode_ranks(const uint8_t* __restrict__ in, Ctrl* c, Desc* desc,
                                                      int32_t* __restrict__ delta, int* status) {
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_w[TILE_WARPS];
    __shared__ unsigned long long s_pre_w;
    if (*status || (c->flags & FLAG_NO_TOPO)) return;
    const Layout lo = c->lo;
    const uint64_t k = c->k_total;
    const unsigned long long rwords = c->rank_words;
    const uint32_t nbd = (uint32_t)cdiv(k, L);
    const uint8_t* widths = in + lo.r2;
    const int32_t* firsts = reinterpret_cast<const int32_t*>(in + lo.r4);
    const uint32_t* pay = reinterpret_cast<const uint32_t*>(in + lo.r5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ntiles = (nbd + TILE_BLOCKS - 1) / TILE_BLOCKS;
    bool corrupt = false;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&c->tile_rdec, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t blk0 = tile * TILE_BLOCKS + warp * BPW;
        uint32_t my_w = 0;
        int32_t my_first = 0;
        if (lane < BPW && blk0 + lane < nbd) {
            my_w = widths[blk0 + lane];
            my_first = firsts[blk0 + lane];
            if (my_w > 32) {
                corrupt = true;
                my_w = 0;
            }
        }
        uint32_t ww = (lane < BPW && my_w) ? 1u + my_w : 0u;
        ww = __reduce_add_sync(FULL, ww);
        if (lane == 0) s_w[warp] = ww;
        __syncthreads();
        if (warp == 0) {
            uint32_t vw = lane < TILE_WARPS ? s_w[lane] : 0, iw = vw;
#pragma unroll
            for (int o = 1; o < TILE_WARPS; o <<= 1) {
                uint32_t t0 = __shfl_up_sync(FULL, iw, o);
                if (lane >= o) iw += t0;
            }
            uint32_t tw = __shfl_sync(FULL, iw, TILE_WARPS - 1);
            unsigned long long pw, pc;
            lookback(desc, tile, tw, 0, pw, pc, status);
            if (lane < TILE_WARPS) s_w[lane] = iw - vw;
            if (lane == 0) {
                s_pre_w = pw;
                if (tile == ntiles - 1 && pw + tw != rwords) set_status(status, ST_CORRUPT);
            }
        }
        __syncthreads();
        unsigned long long woff = s_pre_w + s_w[warp];
#pragma unroll
        for (int j = 0; j < BPW; j++) {
            const uint32_t b = blk0 + j;
            if (b >= nbd) break;
            const uint32_t w = __shfl_sync(FULL, my_w, j);
            const int32_t first = __shfl_sync(FULL, my_first, j);
            int32_t q = first;
            if (w) {
                if (woff + 1 + w <= rwords) q = decode_block(pay, woff, w, first, lane);
                else corrupt = true;
                woff += 1 + w;
            }
            const uint64_t i = (uint64_t)b * 32u + lane;
            if (i < k) delta[i] = q;
        }
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

struct OverrideVal {
    const float* F;
    uint32_t p;
    float v;
    __device__ __forceinline__ float operator()(uint32_t j) const { return j == p ? v : F[j]; }
};

__device__ __forceinline__ int colour_of(const Geo& g, uint32_t x, uint32_t y, uint32_t z) {
    return g.ndim == 2 ? (int)((x + 2u * y) % 5u) : (int)((x + 2u * y + 3u * z) % 7u);
}

// RS^ candidate: returns true and the refined value when accepted.
__device__ bool saddle_candidate(const float* F, const uint32_t* labels, const Geo& g, const Ctrl* c,
                                 uint32_t p, uint32_t x, uint32_t y, uint32_t z, float& vout) {
    const float Fp = F[p];
    GlobalVal val{F};
    // a saddle label is only valid at interior points; anything else is a bad stream
    if (x == 0 || x + 1 >= g.nx || y == 0 || y + 1 >= g.ny || (g.ndim == 3 && (z == 0 || z + 1 >= g.nz)))
        return false;
    if (classify(val, g, p, x, y, z, Fp) == LAB_SAD) return false;   // not lost (any more)
    const uint32_t st[3] = {1u, g.nx, g.nxy};
    float gmin = __int_as_float(0x7F800000);
    for (int ax = 0; ax < g.ndim; ax++) {
        float g1 = fabsf(__fsub_rn(F[p - st[ax]], Fp)), g2 = fabsf(__fsub_rn(F[p + st[ax]], Fp));
        if (g1 > 0.0f && g1 < gmin) gmin = g1;
        if (g2 > 0.0f && g2 < gmin) gmin = g2;
    }
    if (isinf(gmin)) return false;
    // normalised Gaussian kernel over N_r(p) \ {p}, fixed (z, y, x) order
    const int r = c->rbf_k / 2, rz = g.ndim == 3 ? r : 0;
    float num = 0.0f, den = 0.0f;
    for (int dz = -rz; dz <= rz; dz++)
        for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
                const int d2 = dx * dx + dy * dy + dz * dz;
                if (d2 == 0 || d2 > r * r) continue;
                const long long xx = (long long)x + dx, yy = (long long)y + dy, zz = (long long)z + dz;
                if (xx < 0 || yy < 0 || zz < 0 || xx >= g.nx || yy >= g.ny || zz >= g.nz) continue;
                const float gw = c->g_rbf[d2 - 1];
                const float fv = F[(uint32_t)xx + g.nx * ((uint32_t)yy + g.ny * (uint32_t)zz)];
                num = __fadd_rn(num, __fmul_rn(gw, fv));
                den = __fadd_rn(den, gw);
            }
    const float u = __fdiv_rn(num, den);
    const float capv = fminf(__fmul_rn(0.1f, c->h_f), __fmul_rn(0.5f, gmin));
    float stp = __fsub_rn(u, Fp);
    if (stp > capv) stp = capv;
    if (stp < -capv) stp = -capv;
    const float v = __fadd_rn(Fp, stp);
    if (v == Fp) return false;
    OverrideVal nv{F, p, v};
    if (classify(nv, g, p, x, y, z, v) != LAB_SAD) return false;
    for (int ax = 0; ax < g.ndim; ax++) {
        for (int sg = -1; sg <= 1; sg += 2) {
            const uint32_t q = sg < 0 ? p - st[ax] : p + st[ax];
            uint32_t qx = x, qy = y, qz = z;
            if (ax == 0) qx = sg < 0 ? x - 1 : x + 1;
            else if (ax == 1) qy = sg < 0 ? y - 1 : y + 1;
            else qz = sg < 0 ? z - 1 : z + 1;
            const float fq = F[q];
            const int tn = classify(nv, g, q, qx, qy, qz, fq);
            const int to = classify(val, g, q, qx, qy, qz, fq);
            if (tn != to && tn != label_at(labels, q)) return false;
        }
    }
    if (!(fabsf(__fsub_rn(v, Fp)) <= c->h_f)) return false;
    vout = v;
    return true;
}

__global__ void __launch_bounds__(256) k_fixup(const uint8_t* __restrict__ in, Ctrl* c, float* out,
                                               const uint32_t* cp_idx, const int32_t* delta, float* newv,
                                               uint32_t* sad, float* sadv, uint32_t sad_cap, int* status) {
    cg::grid_group grid = cg::this_grid();
    // uniform across the grid: neither word is written by this kernel
    if (*status || (c->flags & FLAG_NO_TOPO)) return;
    const Geo g = c->g;
    const uint32_t* labels = reinterpret_cast<const uint32_t*>(in + c->lo.s6);
    const uint64_t k = c->k_total;
    const float h_f = c->h_f;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    GlobalVal val{out};
    // ---- CP^ + RP^: evaluate every extremum on the QZ^ snapshot (Jacobi)
    unsigned long long restored = 0, skipped = 0;
    for (uint64_t pos = tid; pos < k; pos += nth) {
        const uint32_t p = cp_idx[pos];
        const int lab = label_at(labels, p);
        float nv = __int_as_float(0x7FC00000);
        uint32_t x, y, z;
        coords(g, p, x, y, z);
        const float v0 = out[p];
        if (classify(val, g, p, x, y, z, v0) != lab) {
            const uint32_t st[3] = {1u, g.nx, g.nxy};
            const uint32_t cc[3] = {x, y, z}, dd[3] = {g.nx, g.ny, g.nz};
            float ext = 0.0f;
            bool have = false;
            for (int ax = 0; ax < g.ndim; ax++) {
                if (cc[ax] > 0) {
                    const float u = out[p - st[ax]];
                    if (!have || (lab == LAB_MAX ? u > ext : u < ext)) ext = u;
                    have = true;
                }
                if (cc[ax] + 1 < dd[ax]) {
                    const float u = out[p + st[ax]];
                    if (!have || (lab == LAB_MAX ? u > ext : u < ext)) ext = u;
                    have = true;
                }
            }
            float v;
            const long long dl = delta[pos];
            if (have && step_ulps(ext, lab == LAB_MAX ? dl : -dl, v) && fabsf(__fsub_rn(v, v0)) <= h_f) {
                nv = v;
                restored++;
            } else {
                skipped++;
            }
        }
        newv[pos] = nv;
    }
    grid.sync();
    for (uint64_t pos = tid; pos < k; pos += nth) {
        const float v = newv[pos];
        if (!isnan(v)) out[cp_idx[pos]] = v;
    }
    grid.sync();
    // ---- collect saddles that are still lost (a fixed saddle never breaks again)
    const uint32_t nwords = (g.n + 15) / 16;
    for (uint32_t wi0 = tid - lane; wi0 < nwords; wi0 += nth) {
        const uint32_t wi = wi0 + lane;
        const uint32_t word = wi < nwords ? labels[wi] : 0u;
        uint32_t smask = ((word >> 1) & ~word) & 0x55555555u;   // code 10
        uint32_t lost = 0;
        while (smask) {
            const int bit = __ffs(smask) - 1;
            smask &= smask - 1;
            const uint32_t p = wi * 16u + (uint32_t)(bit >> 1);
            uint32_t x, y, z;
            coords(g, p, x, y, z);
            if (classify(val, g, p, x, y, z, out[p]) != LAB_SAD) lost |= 1u << (bit >> 1);
        }
        const uint32_t cnt = __popc(lost);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        uint32_t base = 0;
        if (lane == 31 && tot) base = atomicAdd(&c->sad_cnt[0], tot);
        base = __shfl_sync(FULL, base, 31);
        uint32_t slot = base + incl - cnt;
        while (lost) {
            const int b = __ffs(lost) - 1;
            lost &= lost - 1;
            if (slot < sad_cap) sad[slot] = wi * 16u + (uint32_t)b;
            slot++;
        }
    }
    (void)lt;
    grid.sync();
    // ---- RS^: colour rounds, two phases each
    const uint32_t ns = min(c->sad_cnt[0], sad_cap);
    const int ncol = g.ndim == 2 ? 5 : 7;
    unsigned long long fixed = 0;
    for (int sw = 0; sw < c->rs_sweeps; sw++) {
        for (int col = 0; col < ncol; col++) {
            for (uint32_t j = tid; j < ns; j += nth) {
                const uint32_t p = sad[j];
                uint32_t x, y, z;
                coords(g, p, x, y, z);
                if (colour_of(g, x, y, z) != col) continue;
                float v;
                sadv[j] = saddle_candidate(out, labels, g, c, p, x, y, z, v) ? v : __int_as_float(0x7FC00000);
            }
            grid.sync();
            for (uint32_t j = tid; j < ns; j += nth) {
                const uint32_t p = sad[j];
                uint32_t x, y, z;
                coords(g, p, x, y, z);
                if (colour_of(g, x, y, z) != col) continue;
                const float v = sadv[j];
                if (!isnan(v)) {
                    out[p] = v;
                    fixed++;
                }
            }
            grid.sync();
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        restored += __shfl_xor_sync(FULL, restored, o);
        skipped += __shfl_xor_sync(FULL, skipped, o);
        fixed += __shfl_xor_sync(FULL, fixed, o);
    }
    if (lane == 0) {
        if (restored) atomicAdd(&c->stat_restored, restored);
        if (skipped) atomicAdd(&c->stat_skipped, skipped);
        if (fixed) atomicAdd(&c->stat_saddle, fixed);
    }
}

// ------------------------------------------------------------ host launchers

void launch_parse_header(const uint8_t* in, uint64_t in_size, uint64_t n_out, Ctrl* c, int* status,
                         cudaStream_t st) {
    k_parse_header<<<1, 32, 0, st>>>(in, in_size, n_out, c, status);
}

void launch_decode_field(const uint8_t* in, Ctrl* c, Desc* desc, float* out, uint32_t* cp_idx,
                         uint32_t ntiles, int sms, int* status, cudaStream_t st) {
    uint32_t grid = hmin<uint32_t>(ntiles, (uint32_t)sms * 6);
    if (grid == 0) grid = 1;
    k_decode_field<<<grid, 256, 0, st>>>(in, c, desc, out, cp_idx, status);
}

void launch_decode_ranks(const uint8_t* in, Ctrl* c, Desc* desc, int32_t* delta, uint32_t max_tiles,
                         int sms, int* status, cudaStream_t st) {
    uint32_t grid = hmin<uint32_t>(max_tiles, (uint32_t)sms * 6);
    if (grid == 0) grid = 1;
    k_decode_ranks<<<grid, 256, 0, st>>>(in, c, desc, delta, status);
}

int fixup_grid(int sms) {
    static int per_sm = -1;
    if (per_sm < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fixup, 256, 0) != cudaSuccess || b < 1)
            b = 1;
        per_sm = b < 4 ? b : 4;
    }
    return per_sm * sms;
}

cudaError_t launch_fixup(const uint8_t* in, Ctrl* c, float* out, const uint32_t* cp_idx,
                         const int32_t* delta, float* newv, uint32_t* sad, float* sadv, uint32_t sad_cap,
                         int sms, int* status, cudaStream_t st) {
    void* args[] = {(void*)&in, (void*)&c, (void*)&out, (void*)&cp_idx, (void*)&delta,
                    (void*)&newv, (void*)&sad, (void*)&sadv, (void*)&sad_cap, (void*)&status};
    return cudaLaunchCooperativeKernel((const void*)k_fixup, dim3(fixup_grid(sms)), dim3(256), args, 0, st);
}

}  // namespace tsz
