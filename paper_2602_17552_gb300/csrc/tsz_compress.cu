// tsz_compress.cu -- compression kernels (Section IV-A of arXiv 2602.17552).
//
// Pipeline on one stream:
//   k_range_cd_col / _vec / k_range_cd
//                   one read of the field: value range (min, max), finite
//                   check and, unless NO_TOPO, the CD labels written straight
//                   into section (6) (the column form walks z with rows
//                   z - 1, z, z + 1 in registers)
//   k_qparams       one thread: eps, bin width w, its reciprocal r, half-width h
//   k_bm_zero       the rank mode (key bitmaps or radix sort) and zeroed bitmaps
//   k_encode_field  one read of field + labels per 8192-point tile: QZ, B + LZ,
//                   BE into the tile's payload slot; extrema keys to two lists
//                   (and their bits to the key bitmaps)
//   k_enc_tile_scan, k_enc_copy
//                   slice-parallel scan of the tile counts, slots to the stream
//   k_bm_sums, k_bm_prefix, k_bin_table, k_rank_delta
//                   dense rank per (type, bin) = RP's delta from the bitmaps,
//                   or, when the key span does not fit, the radix sort
//                   (k_os_*: LSD passes of <= 9-bit digits) and k_rank_*
//   k_encode_ranks, k_rank_tile_scan, k_rank_copy
//                   the same codec on the delta sequence (no QZ)
//   k_finalize      header, section padding, stream size
#include "tsz_internal.h"

namespace tsz {

// ================================================================ range + CD

// One warp owns chunks of 512 consecutive points: lane l handles points
// base + 32k + l (k = 0..15), so every load is a coalesced 128-byte row; the
// 2-bit labels of 32 points are gathered with two ballots and interleaved into
// two label words.
template <bool TOPO, bool COUNTS, bool STATS>
__global__ void __launch_bounds__(256) k_range_cd(const float* __restrict__ a, const Geo g, Ctrl* c,
                                                  uint32_t* __restrict__ labels,
                                                  unsigned long long* counts) {
    griddep_enter();
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = (g.n + 511) / 512;
    const uint32_t nwords = (g.n + 15) / 16;
    const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t kmin = 0, kmax = 0;   // min as max of ~key
    bool bad = false;
    unsigned long long cm = 0, cs = 0, cM = 0;
    uint32_t sad_cnt = 0;
    GlobalVal val{a};
    for (uint32_t ch = warp0; ch < nchunks; ch += nwarps) {
        const uint32_t base = ch * 512u;
        uint32_t x, y, z;
        uint32_t i0 = base + lane;
        coords(g, i0 < g.n ? i0 : 0, x, y, z);
        uint32_t word = 0;
#pragma unroll 4
        for (int k = 0; k < 16; k++) {
            const uint32_t i = base + 32u * k + lane;
            int lab = 0;
            if (i < g.n) {
                float v = __ldg(a + i);
                if (!isfinite(v)) bad = true;
                uint32_t key = ord_key(v);
                kmax = max(kmax, key);
                kmin = max(kmin, ~key);
                if (TOPO) lab = classify(val, g, i, x, y, z, v);
            }
            if (TOPO) {
                uint32_t b0 = __ballot_sync(FULL, lab & 1);
                uint32_t b1 = __ballot_sync(FULL, lab >> 1);
                if (lane == 2 * k) word = spread16(b0) | (spread16(b1) << 1);
                if (lane == 2 * k + 1) word = spread16(b0 >> 16) | (spread16(b1 >> 16) << 1);
            }
            x += 32;
            while (x >= g.nx) {
                x -= g.nx;
                if (++y == g.ny) { y = 0; ++z; }
            }
        }
        if (TOPO) {
            uint32_t wi = ch * 32u + lane;
            if (wi < nwords) {
                if (labels) labels[wi] = word;
                if (STATS) sad_cnt += __popc((word >> 1) & ~word & 0x55555555u);
                if (COUNTS) {
                    uint32_t lo = word & 0x55555555u, hi = (word >> 1) & 0x55555555u;
                    cm += __popc(lo & ~hi);
                    cs += __popc(hi & ~lo);
                    cM += __popc(lo & hi);
                }
            }
        }
    }
    // reduce and publish
    kmax = __reduce_max_sync(FULL, kmax);
    kmin = __reduce_max_sync(FULL, kmin);
    bool anybad = __any_sync(FULL, bad);
    const uint32_t sad_tot = __reduce_add_sync(FULL, sad_cnt);
    if (STATS && lane == 0) {
        if (kmax) atomicMax(&c->max_key, kmax);
        if (kmin) atomicMax(&c->min_inv, kmin);
        if (anybad) atomicExch(&c->nonfinite, 1u);
        if (sad_tot) atomicAdd(&c->k_sad, (unsigned long long)sad_tot);
    }
    if (COUNTS) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cm += __shfl_xor_sync(FULL, cm, o);
            cs += __shfl_xor_sync(FULL, cs, o);
            cM += __shfl_xor_sync(FULL, cM, o);
        }
        if (lane == 0) {
            if (cm) atomicAdd(&counts[1], cm);
            if (cs) atomicAdd(&counts[2], cs);
            if (cM) atomicAdd(&counts[3], cM);
        }
    }
}

// ------------------------------------------------- range + CD, vector path
//
// For nx % 4 == 0 (rows start on 16-byte boundaries): lane l of a warp owns
// the quad of points [4q, 4q+4) of a 128-point chunk, so the field, the rows
// above/below and the planes before/after are single float4 loads, and the x
// neighbours of a quad come from the adjacent lanes by shuffle.  Points in rows
// with all y/z neighbours present take a branch-free comparison path; boundary
// rows fall back to the general rule.  Coordinates advance by the grid stride
// without divisions.

// NaN-propagating minimum / maximum (PTX min.NaN / max.NaN): a comparison
// against a NaN result is false, exactly as for the strict comparisons of the
// rule itself, so "both neighbours higher" == (min(a, b) > v) for any input.
__device__ __forceinline__ float min_nan(float a, float b) {
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float max_nan(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Section IV-A(1) at a point whose y (and z) pairs exist: per axis, H = both
// neighbours higher, L = both lower; m = all H, M = all L, s = every axis H or
// L with at least one of each.  An absent x neighbour is passed as the other
// one (`xl` / `xr` false), which leaves H and L of the axis to the neighbour
// that exists and rules out a saddle.
__device__ __forceinline__ uint32_t cd_fast(float v, float l, float r, bool xl, bool xr, float ym, float yp,
                                            float zm, float zp, bool three) {
    const float a = xl ? l : r, b = xr ? r : l;
    const bool Hx = min_nan(a, b) > v, Lx = max_nan(a, b) < v;
    const bool Hy = min_nan(ym, yp) > v, Ly = max_nan(ym, yp) < v;
    const bool Hz = !three || min_nan(zm, zp) > v, Lz = !three || max_nan(zm, zp) < v;
    const bool m = Hx && Hy && Hz, M = Lx && Ly && Lz;
    const bool s = xl && xr && (Hx || Lx) && (Hy || Ly) && (Hz || Lz) && !m && !M;
    return (uint32_t)(m | M) | ((uint32_t)(s | M) << 1);
}

// cd_fast() for finite values, with the comparisons on the FMA pipe: for
// finite u != v, fl(u - v) is nonzero with the sign of u - v (no flush to
// zero, overflow keeps the sign) and fl(v - v) = +0, so with -0 folded to +0
// beforehand (cz4) bit 31 of fl(u - v) is u < v.  The per-axis tests are then bitwise ANDs of sign words.  Used by
// the compression pass only, where a non-finite field is rejected anyway.
__device__ __forceinline__ uint32_t lt_bit(float u, float v) { return __float_as_uint(__fsub_rn(u, v)); }
__device__ __forceinline__ float4 cz4(float4 v) {
    return make_float4(__fadd_rn(v.x, 0.0f), __fadd_rn(v.y, 0.0f), __fadd_rn(v.z, 0.0f), __fadd_rn(v.w, 0.0f));
}

template <bool THREE>
__device__ __forceinline__ uint32_t cd_sign(float v, float l, float r, bool xl, bool xr, float ym, float yp,
                                            float zm, float zp) {
    const float a = xl ? l : r, b = xr ? r : l;
    const uint32_t Lx = lt_bit(a, v) & lt_bit(b, v), Hx = lt_bit(v, a) & lt_bit(v, b);
    const uint32_t Ly = lt_bit(ym, v) & lt_bit(yp, v), Hy = lt_bit(v, ym) & lt_bit(v, yp);
    const uint32_t Lz = THREE ? lt_bit(zm, v) & lt_bit(zp, v) : 0x80000000u;
    const uint32_t Hz = THREE ? lt_bit(v, zm) & lt_bit(v, zp) : 0x80000000u;
    const uint32_t m = Hx & Hy & Hz, M = Lx & Ly & Lz;
    uint32_t s = (Hx | Lx) & (Hy | Ly) & (Hz | Lz) & ~m & ~M;
    if (!(xl && xr)) s = 0u;
    return ((m | M) >> 31) | (((s | M) >> 31) << 1);
}

template <bool TOPO, bool COUNTS, bool STATS, bool THREE>
__global__ void __launch_bounds__(512) k_range_cd_vec(const float* __restrict__ a, const Geo g, Ctrl* c,
                                                      uint32_t* __restrict__ labels,
                                                      unsigned long long* counts) {
    griddep_enter();
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = (g.n + 127) / 128;
    const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    constexpr bool three = THREE;
    // coordinates of this lane's first quad, and the grid stride in (x, y, z) digits
    uint32_t x, y, z;
    {
        const uint64_t i0 = (uint64_t)warp0 * 128 + 4u * lane;
        coords(g, i0 < g.n ? (uint32_t)i0 : 0u, x, y, z);
    }
    const uint64_t S = (uint64_t)nwarps * 128;
    const uint32_t sx = (uint32_t)(S % g.nx);
    const uint64_t sr = S / g.nx;
    const uint32_t sy = (uint32_t)(sr % g.ny);
    const uint32_t sz = (uint32_t)(sr / g.ny);
    float vmin = __int_as_float(0x7F800000), vmax = __int_as_float(0xFF800000);
    float fin = 0.0f;   // sum of (v - v): +0 while every value is finite, NaN after an inf or NaN
    unsigned long long cm = 0, cs = 0, cM = 0;
    GlobalVal val{a};
    for (uint32_t ch = warp0; ch < nchunks; ch += nwarps) {
        const uint32_t i0 = ch * 128u + 4u * lane;
        const bool active = i0 < g.n;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active) v = __ldg(reinterpret_cast<const float4*>(a + i0));
        if (STATS && active) {
            vmin = fminf(fminf(vmin, v.x), fminf(v.y, fminf(v.z, v.w)));
            vmax = fmaxf(fmaxf(vmax, v.x), fmaxf(v.y, fmaxf(v.z, v.w)));
            fin = __fadd_rn(fin, __fadd_rn(__fadd_rn(__fsub_rn(v.x, v.x), __fsub_rn(v.y, v.y)),
                                           __fadd_rn(__fsub_rn(v.z, v.z), __fsub_rn(v.w, v.w))));
        }
        if (TOPO) {
            float left = __shfl_up_sync(FULL, v.w, 1);
            float right = __shfl_down_sync(FULL, v.x, 1);
            const bool xl = x > 0, xr = x + 4 < g.nx;
            if (active && lane == 0 && xl) left = __ldg(a + i0 - 1);
            if (active && lane == 31 && xr) right = __ldg(a + i0 + 4);
            uint32_t bits = 0;
            if (active) {
                const bool inner = y > 0 && y + 1 < g.ny && (!three || (z > 0 && z + 1 < g.nz));
                if (inner) {
                    const float4 ym = __ldg(reinterpret_cast<const float4*>(a + i0 - g.nx));
                    const float4 yp = __ldg(reinterpret_cast<const float4*>(a + i0 + g.nx));
                    float4 zm = ym, zp = yp;
                    if (three) {
                        zm = __ldg(reinterpret_cast<const float4*>(a + i0 - g.nxy));
                        zp = __ldg(reinterpret_cast<const float4*>(a + i0 + g.nxy));
                    }
                    if (STATS) {
                        // -0 - (+0) = -0 would read as "less": fold every -0 to +0 first
                        const float4 c = cz4(v), cym = cz4(ym), cyp = cz4(yp);
                        const float4 czm = THREE ? cz4(zm) : cym, czp = THREE ? cz4(zp) : cyp;
                        const float cl = __fadd_rn(left, 0.0f), cr = __fadd_rn(right, 0.0f);
                        bits = cd_sign<THREE>(c.x, cl, c.y, xl, true, cym.x, cyp.x, czm.x, czp.x) |
                               cd_sign<THREE>(c.y, c.x, c.z, true, true, cym.y, cyp.y, czm.y, czp.y) << 2 |
                               cd_sign<THREE>(c.z, c.y, c.w, true, true, cym.z, cyp.z, czm.z, czp.z) << 4 |
                               cd_sign<THREE>(c.w, c.z, cr, true, xr, cym.w, cyp.w, czm.w, czp.w) << 6;
                    } else
                        bits = cd_fast(v.x, left, v.y, xl, true, ym.x, yp.x, zm.x, zp.x, three) |
                               cd_fast(v.y, v.x, v.z, true, true, ym.y, yp.y, zm.y, zp.y, three) << 2 |
                               cd_fast(v.z, v.y, v.w, true, true, ym.z, yp.z, zm.z, zp.z, three) << 4 |
                               cd_fast(v.w, v.z, right, true, xr, ym.w, yp.w, zm.w, zp.w, three) << 6;
                } else {
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        bits |= (uint32_t)classify(val, g, i0 + j, x + j, y, z, vv[j]) << (2 * j);
                }
            }
            // four lanes make one 16-point label word
            const uint32_t b1 = __shfl_down_sync(FULL, bits, 1);
            const uint32_t b2 = __shfl_down_sync(FULL, bits, 2);
            const uint32_t b3 = __shfl_down_sync(FULL, bits, 3);
            if (active && (lane & 3) == 0) {
                const uint32_t word = bits | (b1 << 8) | (b2 << 16) | (b3 << 24);
                if (labels) labels[i0 >> 4] = word;
                if (STATS) cs += __popc((word >> 1) & ~word & 0x55555555u);
                if (COUNTS) {
                    const uint32_t lo = word & 0x55555555u, hi = (word >> 1) & 0x55555555u;
                    cm += __popc(lo & ~hi);
                    cs += __popc(hi & ~lo);
                    cM += __popc(lo & hi);
                }
            }
        }
        // advance by the grid stride
        x += sx;
        uint32_t cy = 0;
        if (x >= g.nx) { x -= g.nx; cy = 1; }
        y += sy + cy;
        uint32_t cz = 0;
        if (y >= g.ny) { y -= g.ny; cz = 1; }
        z += sz + cz;
    }
    if (STATS) {
        uint32_t kmax = vmax >= vmin ? ord_key(vmax) : 0u;
        uint32_t kmin = vmax >= vmin ? ~ord_key(vmin) : 0u;
        kmax = __reduce_max_sync(FULL, kmax);
        kmin = __reduce_max_sync(FULL, kmin);
        const bool anybad = __any_sync(FULL, isnan(fin));
        const unsigned long long sad = TOPO ? __reduce_add_sync(FULL, (uint32_t)cs) : 0u;
        if (lane == 0) {
            if (kmax) atomicMax(&c->max_key, kmax);
            if (kmin) atomicMax(&c->min_inv, kmin);
            if (anybad) atomicExch(&c->nonfinite, 1u);
            if (sad) atomicAdd(&c->k_sad, sad);
        }
    }
    if (COUNTS) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cm += __shfl_xor_sync(FULL, cm, o);
            cs += __shfl_xor_sync(FULL, cs, o);
            cM += __shfl_xor_sync(FULL, cM, o);
        }
        if (lane == 0) {
            if (cm) atomicAdd(&counts[1], cm);
            if (cs) atomicAdd(&counts[2], cs);
            if (cM) atomicAdd(&counts[3], cM);
        }
    }
}

// The compression pass for 3D fields whose planes hold a whole number of
// 128-point chunks: a warp walks one chunk position down z (a segment of zseg
// planes) and keeps the rows z-1, z, z+1 in registers, so each value comes
// from DRAM about once (the y-neighbour rows are the neighbouring warps'
// rows, read from L2).  Same results as k_range_cd_vec.  The segment is
// CD_ZSEG planes, shorter when the field has too few columns to give every
// SM enough warps (each segment reads two planes more than it labels).
constexpr uint32_t CD_ZSEG = 32, CD_ZSEG_MIN = 4;

__global__ void __launch_bounds__(256) k_range_cd_col(const float* __restrict__ a, const Geo g, Ctrl* c,
                                                      uint32_t* __restrict__ labels, uint32_t zseg) {
    griddep_enter();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t ncols = g.nxy / 128, nsegs = (g.nz + zseg - 1) / zseg;
    float vmin = __int_as_float(0x7F800000), vmax = __int_as_float(0xFF800000);
    float fin = 0.0f;   // sum of (v - v): +0 while every value is finite, NaN after an inf or NaN
    uint32_t cs = 0;
    GlobalVal val{a};
    for (uint32_t wi = gw; wi < ncols * nsegs; wi += nw) {
        const uint32_t col = wi % ncols, seg = wi / ncols;
        const uint32_t p0 = col * 128u + 4u * lane;   // this lane's quad within a plane
        const uint32_t t = fdiv(p0, g.fx);
        const uint32_t x = p0 - t * g.nx, y = t;       // one plane: t < ny
        const bool xl = x > 0, xr = x + 4 < g.nx, yin = y > 0 && y + 1 < g.ny;
        const uint32_t z0 = seg * zseg, z1 = min(g.nz, z0 + zseg);
        const float4* a4 = reinterpret_cast<const float4*>(a);
        float4 prev = make_float4(0.f, 0.f, 0.f, 0.f);
        if (z0 > 0) prev = __ldg(a4 + ((size_t)(z0 - 1) * g.nxy + p0) / 4);
        float4 cur = __ldg(a4 + ((size_t)z0 * g.nxy + p0) / 4);
        for (uint32_t z = z0; z < z1; z++) {
            const uint32_t i0 = z * g.nxy + p0;
            float4 next = make_float4(0.f, 0.f, 0.f, 0.f);
            if (z + 1 < g.nz) next = __ldg(a4 + (i0 + g.nxy) / 4);
            const float4 v = cur;
            vmin = fminf(fminf(vmin, v.x), fminf(v.y, fminf(v.z, v.w)));
            vmax = fmaxf(fmaxf(vmax, v.x), fmaxf(v.y, fmaxf(v.z, v.w)));
            fin = __fadd_rn(fin, __fadd_rn(__fadd_rn(__fsub_rn(v.x, v.x), __fsub_rn(v.y, v.y)),
                                           __fadd_rn(__fsub_rn(v.z, v.z), __fsub_rn(v.w, v.w))));
            float left = __shfl_up_sync(FULL, v.w, 1);
            float right = __shfl_down_sync(FULL, v.x, 1);
            if (lane == 0 && xl) left = __ldg(a + i0 - 1);
            if (lane == 31 && xr) right = __ldg(a + i0 + 4);
            uint32_t bits = 0;
            if (yin && z > 0 && z + 1 < g.nz) {
                const float4 ym = __ldg(a4 + (i0 - g.nx) / 4);
                const float4 yp = __ldg(a4 + (i0 + g.nx) / 4);
                // -0 - (+0) = -0 would read as "less": fold every -0 to +0 first
                const float4 cv = cz4(v), cym = cz4(ym), cyp = cz4(yp), czm = cz4(prev), czp = cz4(next);
                const float cl = __fadd_rn(left, 0.0f), cr = __fadd_rn(right, 0.0f);
                bits = cd_sign<true>(cv.x, cl, cv.y, xl, true, cym.x, cyp.x, czm.x, czp.x) |
                       cd_sign<true>(cv.y, cv.x, cv.z, true, true, cym.y, cyp.y, czm.y, czp.y) << 2 |
                       cd_sign<true>(cv.z, cv.y, cv.w, true, true, cym.z, cyp.z, czm.z, czp.z) << 4 |
                       cd_sign<true>(cv.w, cv.z, cr, true, xr, cym.w, cyp.w, czm.w, czp.w) << 6;
            } else {
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; j++) bits |= (uint32_t)classify(val, g, i0 + j, x + j, y, z, vv[j]) << (2 * j);
            }
            // four lanes make one 16-point label word
            const uint32_t b1 = __shfl_down_sync(FULL, bits, 1);
            const uint32_t b2 = __shfl_down_sync(FULL, bits, 2);
            const uint32_t b3 = __shfl_down_sync(FULL, bits, 3);
            if ((lane & 3) == 0) {
                const uint32_t word = bits | (b1 << 8) | (b2 << 16) | (b3 << 24);
                labels[i0 >> 4] = word;
                cs += __popc((word >> 1) & ~word & 0x55555555u);
            }
            prev = cur;
            cur = next;
        }
    }
    uint32_t kmax = vmax >= vmin ? ord_key(vmax) : 0u;
    uint32_t kmin = vmax >= vmin ? ~ord_key(vmin) : 0u;
    kmax = __reduce_max_sync(FULL, kmax);
    kmin = __reduce_max_sync(FULL, kmin);
    const bool anybad = __any_sync(FULL, isnan(fin));
    const uint32_t sad = __reduce_add_sync(FULL, cs);
    if (lane == 0) {
        if (kmax) atomicMax(&c->max_key, kmax);
        if (kmin) atomicMax(&c->min_inv, kmin);
        if (anybad) atomicExch(&c->nonfinite, 1u);
        if (sad) atomicAdd(&c->k_sad, (unsigned long long)sad);
    }
}

// counts[0] = n - (m + s + M)
__global__ void k_count_regular(uint32_t n, unsigned long long* counts) {
    griddep_enter();
    counts[0] = (unsigned long long)n - counts[1] - counts[2] - counts[3];
}

// ============================================================ quantiser setup

// Section II-C, with a quantiser provable in binary32: eps from the bound mode;
// bins of width w = 2h, h = eps - (M + eps) 2^-21 so the binary32 round trip
// stays within eps; constant fields are coded exactly.
__global__ void k_qparams(Ctrl* c, int* status) {
    griddep_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (c->nonfinite) {
        set_status(status, ST_NONFINITE);
        return;
    }
    float vmin = key_float(~c->min_inv);
    float vmax = key_float(c->max_key);
    c->vmin = vmin;
    c->vmax = vmax;
    double eps = c->rel ? __dmul_rn(c->eb, __dsub_rn((double)vmax, (double)vmin)) : c->eb;
    c->eps = eps;
    if (vmax == vmin) {
        float w = (vmin == 0.0f) ? 1.0f : fabsf(vmin);
        c->const_field = 1;
        c->w_f = w;
        c->r_f = __double2float_rn(__ddiv_rn(1.0, (double)w));
        c->h_f = 0.0f;
        return;
    }
    if (!(eps > 0.0) || !isfinite(eps)) {
        set_status(status, ST_EB_SMALL);
        return;
    }
    double M = fmax(fabs((double)vmin), fabs((double)vmax));
    double h = __dsub_rn(eps, __dmul_rn(__dadd_rn(M, eps), 0x1p-21));
    if (!(h >= __dmul_rn(eps, 0.5))) {
        set_status(status, ST_EB_SMALL);
        return;
    }
    if (!(__dmul_rn(2.0, h) <= (double)3.0e38f)) {
        set_status(status, ST_INVALID);
        return;
    }
    float w = __double2float_rd(__dmul_rn(2.0, h));
    c->w_f = w;
    c->r_f = __double2float_rn(__ddiv_rn(1.0, (double)w));
    c->h_f = __double2float_rd(h);
}

// ====================================================================== codec
//
// B + LZ + BE (Sections II-C, IV-A): block b holds codes q[32b .. 32b+31] (the
// tail block repeats its last code); Lorenzo residuals d_0 = 0,
// d_j = q_j - q_{j-1}; w_b = bit length of max|d|; w_b = 0 is a constant block.
// A non-constant block stores a sign plane and w_b magnitude planes, one
// ballot each, at its exclusive prefix offset in the payload section.

struct EncOut {
    uint32_t* cbits;
    uint8_t* width;
    int32_t* first;
    uint32_t* pay;
};

// Field encoder, one 8192-point tile (256 blocks) per CTA, one block per
// thread.  The tile's values are staged in shared memory with coalesced
// 16-byte loads (rows padded to 36 words, so a thread's row reads are
// conflict-free); each thread then quantises its 32 values, forms the Lorenzo
// residuals, the width and the sign plane, and builds its magnitude planes
// with register bit operations (one instruction handles a bit of one block's
// element, as a ballot would, without moving bits between lanes).  The packed
// payload of the tile goes to its fixed-size slot of a scratch area; no CTA
// waits for another: the tile prefixes come from a scan afterwards
// (k_enc_tile_scan) and k_enc_copy moves every slot to its place in the
// payload section.  TOPO also reads the labels and appends (key,
// tile << 13 | index of the extremum within its tile) pairs to the maxima /
// minima lists; the rank scatter turns the pair into the extremum's position
// in the delta sequence.
constexpr int ENC_ROW = 36;                          // shared words per staged block row
constexpr int TILE_PAY = ENC_TILE_BLOCKS * 33;       // worst-case payload words of a tile: its slot
constexpr int TILE_POS_BITS = 13;                    // 8192 points per tile
static_assert(ENC_TILE_BLOCKS * 32 == (1 << TILE_POS_BITS), "tile size");
static_assert(ENC_TILE_BLOCKS * ENC_ROW >= TILE_PAY, "payload staging");

//
// CODEC = false (format v2, whose payload k_encode_tiles writes): the same
// pass over the linear tiles without the payload -- the extremum lists, the
// tile's extremum count, and the residual sum of the RBF parameters (always
// that of blocks of 32 consecutive points).  The grid may then hold more
// CTAs than linear tiles (as many as the format's payload tiles): those only
// zero their count.
template <bool TOPO, bool CODEC>
__global__ void __launch_bounds__(256, 4) k_encode_field(const float* __restrict__ a,
                                                         const uint32_t* __restrict__ labels, Ctrl* c,
                                                         uint2* tcnt, EncOut o, uint2* listM, uint2* listm,
                                                         uint32_t* region, int* status) {
    griddep_enter();
    __shared__ __align__(16) uint32_t s_buf[ENC_TILE_BLOCKS * ENC_ROW];
    __shared__ uint32_t s_wsum[8][3];
    __shared__ uint32_t s_base[2];
    __shared__ uint32_t s_ext[8][2];
    __shared__ unsigned long long s_sum;
    if (*status) return;
    const uint32_t n = c->g.n, nb = c->g.nb;
    const float r = c->r_f;
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t tile = blockIdx.x;
    const uint32_t b = tile * ENC_TILE_BLOCKS + t;   // this thread's block
    const uint64_t p0 = (uint64_t)tile * (ENC_TILE_BLOCKS * 32);
    if (!CODEC && p0 >= n) {
        if (t == 0) tcnt[tile] = make_uint2(0u, 0u);
        return;
    }
    const uint64_t left = (uint64_t)n - p0;
    const uint32_t npts = left < (uint64_t)(ENC_TILE_BLOCKS * 32) ? (uint32_t)left : (uint32_t)(ENC_TILE_BLOCKS * 32);
    if (t == 0) s_sum = 0;
    // ---- stage the tile's values
    if (npts == ENC_TILE_BLOCKS * 32 && (reinterpret_cast<uintptr_t>(a) & 15u) == 0) {
        const float4* src = reinterpret_cast<const float4*>(a + p0);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t idx = k * 256 + t;   // float4 index within the tile
            const float4 v = __ldcs(src + idx);
            *reinterpret_cast<float4*>(s_buf + (idx >> 3) * ENC_ROW + (idx & 7) * 4) = v;
        }
    } else {
        for (uint32_t i = t; i < npts; i += 256) s_buf[(i >> 5) * ENC_ROW + (i & 31)] = __float_as_uint(__ldcs(a + p0 + i));
    }
    uint2 lw = make_uint2(0u, 0u);
    if (TOPO && b < nb) lw = reinterpret_cast<const uint2*>(labels)[b];
    uint32_t xmM = 0, xmm = 0;   // extremum masks (bit e: element e), maxima / minima
    if (TOPO) {
        const uint32_t lo0 = lw.x & 0x55555555u, hi0 = (lw.x >> 1) & 0x55555555u;
        const uint32_t lo1 = lw.y & 0x55555555u, hi1 = (lw.y >> 1) & 0x55555555u;
        const uint32_t valid = b < nb ? (n - b * 32u >= 32u ? FULL : (1u << (n - b * 32u)) - 1u) : 0u;
        xmM = (compact16(lo0 & hi0) | compact16(lo1 & hi1) << 16) & valid;    // M = 11
        xmm = (compact16(lo0 & ~hi0) | compact16(lo1 & ~hi1) << 16) & valid;  // m = 01
        // the tile's extremum counts are known from the labels alone: their list
        // ranges are reserved now, so that the atomics' round trip overlaps the
        // block codec instead of holding the whole CTA later
        const uint32_t cMw = __reduce_add_sync(FULL, __popc(xmM)), cmw = __reduce_add_sync(FULL, __popc(xmm));
        if (lane == 0) {
            s_ext[warp][0] = cMw;
            s_ext[warp][1] = cmw;
        }
    }
    __syncthreads();
    uint32_t r_base0 = 0, r_base1 = 0;   // thread 0: the reserved list offsets, stored before the scan
    if (TOPO && t == 0) {
        uint32_t eM = 0, em = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            eM += s_ext[k][0];
            em += s_ext[k][1];
        }
        r_base0 = eM ? atomicAdd(&c->cnt_max, eM) : 0u;
        r_base1 = em ? atomicAdd(&c->cnt_min, em) : 0u;
    }
    // ---- this thread's block: codes, residuals, width, sign plane
    uint32_t m[32];
    uint32_t sgn = 0, orr = 0, sum = 0;
    int32_t first = 0;
    if (b < nb) {
        const uint32_t* row = s_buf + t * ENC_ROW;
        const uint32_t nvalid = min(32u, n - b * 32u);
        int32_t prev = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint4 v4 = *reinterpret_cast<const uint4*>(row + 4 * k);
            const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int e = 4 * k + j;
                int32_t q = quantize(__uint_as_float(vv[j]), r);
                if (e > 0 && (uint32_t)e >= nvalid) q = prev;   // the tail block repeats its last code
                const int32_t d = e ? q - prev : 0;
                if (e == 0) first = q;
                if (d < 0) sgn |= 1u << e;
                m[e] = (uint32_t)(d < 0 ? -d : d);
                orr |= m[e];
                sum += m[e];
                prev = q;
            }
        }
    }
    const uint32_t w = 32u - __clz(orr);   // bit length of max |d|
    const uint32_t W = __reduce_max_sync(FULL, w);   // the warp's widest block: picks the transpose
    const uint32_t words = (CODEC && b < nb && w) ? 1u + w : 0u;
    if (TOPO && t == 0) {   // read after the scan's barrier
        s_base[0] = r_base0;
        s_base[1] = r_base1;
    }
    // ---- exclusive prefixes over the tile's blocks: payload words, maxima, minima
    uint32_t iw = words, iM = __popc(xmM), im = __popc(xmm);
#pragma unroll
    for (int of = 1; of < 32; of <<= 1) {
        const uint32_t a0 = __shfl_up_sync(FULL, iw, of), a1 = __shfl_up_sync(FULL, iM, of),
                       a2 = __shfl_up_sync(FULL, im, of);
        if (lane >= (uint32_t)of) { iw += a0; iM += a1; im += a2; }
    }
    if (lane == 31) { s_wsum[warp][0] = iw; s_wsum[warp][1] = iM; s_wsum[warp][2] = im; }
    {
        unsigned long long sa = sum;
#pragma unroll
        for (int of = 16; of > 0; of >>= 1) sa += __shfl_xor_sync(FULL, sa, of);
        if (lane == 0 && sa) atomicAdd(&s_sum, sa);
    }
    __syncthreads();
    uint32_t ow = 0, oM = 0, om = 0, tw = 0, tM = 0, tm = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const uint32_t v0 = s_wsum[k][0], v1 = s_wsum[k][1], v2 = s_wsum[k][2];
        if (k < (int)warp) { ow += v0; oM += v1; om += v2; }
        tw += v0; tM += v1; tm += v2;
    }
    ow += iw - words;
    oM += iM - __popc(xmM);
    om += im - __popc(xmm);
    if (t == 0) {
        tcnt[tile] = make_uint2(tw, tM + tm);
        unsigned long long* sl = c->sl_tile[tile / slice_len(gridDim.x)];
        if (tw) atomicAdd(sl, (unsigned long long)tw);
        if (tM + tm) atomicAdd(sl + 1, (unsigned long long)(tM + tm));
        if (s_sum) atomicAdd(&c->sum_abs, s_sum);
    }
    if (TOPO) {
        // (key, position) pairs of this block's extrema, in index order; with
        // the bitmap ranks also each key's bit in its list's bitmap
        const uint32_t* row = s_buf + t * ENC_ROW;
        uint32_t* bmM = nullptr;
        uint32_t* bmm = nullptr;
        uint32_t baseM = 0, basem = 0;
        if (c->rank_bitmap) {
            const uint32_t W = c->bm_words;
            bmM = region + c->bm_off;
            bmm = bmM + (size_t)W;
            baseM = ~c->min_inv;   // ord(vmin): the smallest maximum key
            basem = ~c->max_key;   // ~ord(vmax): the smallest minimum key
        }
        uint32_t oMg = s_base[0] + oM, omg = s_base[1] + om, local = oM + om;
        uint32_t xm = xmM | xmm;
        while (xm) {
            const int e = __ffs(xm) - 1;
            xm &= xm - 1;
            const uint32_t key = ord_key(__uint_as_float(row[e]));
            const uint32_t pos = tile << TILE_POS_BITS | local++;
            if ((xmM >> e) & 1u) {
                listM[oMg++] = make_uint2(key, pos);
                if (bmM) {
                    const uint32_t rel = key - baseM;
                    atomicOr(bmM + (rel >> 5), 1u << (rel & 31));
                }
            } else {
                listm[omg++] = make_uint2(~key, pos);
                if (bmm) {
                    const uint32_t rel = ~key - basem;
                    atomicOr(bmm + (rel >> 5), 1u << (rel & 31));
                }
            }
        }
    }
    if (!CODEC) return;
    __syncthreads();   // the staged values are no longer read: the buffer takes the payload
    if (words) {
        uint32_t* dst = s_buf + ow;
        dst[0] = sgn;
        values_to_planes(W, w, m, [&](int r, uint32_t pl) { dst[1 + r] = pl; });
    }
    if (b < nb) {
        o.width[b] = (uint8_t)w;
        o.first[b] = first;
    }
    {   // constant-block bits: one word per warp of blocks
        const uint32_t cb = __ballot_sync(FULL, b < nb && w == 0);
        if (lane == 0 && (b >> 5) < (nb + 31) / 32) o.cbits[b >> 5] = cb;
    }
    __syncthreads();
    uint32_t* slot = o.pay + (size_t)tile * TILE_PAY;
    for (uint32_t k = t; k < tw; k += 256) slot[k] = s_buf[k];
}

// Format v2 field encoder (tile-shaped blocks, Section II-C's B + LZ + BE on
// 8 x 4 / 4 x 4 x 2 tiles): one payload tile of 256 blocks per CTA, one block
// per thread.  The block's 32 values are read from the field (positions
// outside the domain take the nearest inside point, each coordinate
// clamped) and quantised; q' = q - q_0.  Two residual sets, in 32-bit
// modular arithmetic: the chain in element order, d_e = q'_e - q'_{e-1},
// and the block-local Lorenzo differences (inclusion-exclusion over the
// preceding corners, q' = 0 outside the block).  The one with the smaller
// widest residual is coded (Lorenzo only when strictly smaller), its choice
// in bit 7 of the width byte; sign and magnitude planes as in format v1.
// The payload goes to the tile's scratch slot and the tile's word count to
// tcnt[tile].x; the linear pass (CODEC = false) has written .y already.
template <int ND>
__global__ void __launch_bounds__(256, 4) k_encode_tiles(const float* __restrict__ a, Ctrl* c, uint2* tcnt,
                                                         EncOut o, int* status) {
    griddep_enter();
    using TS = TileShape<ND>;
    constexpr uint32_t BX = TS::BX, BY = TS::BY, BZ = TS::BZ;
    __shared__ __align__(16) uint32_t s_buf[TILE_PAY];
    __shared__ uint32_t s_wsum[8];
    if (*status) return;
    const Geo g = c->g;
    const uint32_t nbf = c->nb_fmt;
    const float r = c->r_f;
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t tile = blockIdx.x;
    const uint32_t b = tile * ENC_TILE_BLOCKS + t;
    uint32_t mag[32];
    uint32_t sgn = 0, w = 0, sel = 0;
    int32_t first = 0;
    if (b < nbf) {
        const uint32_t nbx = (g.nx + BX - 1) / BX, nby = (g.ny + BY - 1) / BY;
        const uint32_t gx = b % nbx, gy = (b / nbx) % nby, gz = b / (nbx * nby);
        uint32_t qp[32];
#pragma unroll
        for (int e = 0; e < 32; e++) {
            const uint32_t x = min(gx * BX + (uint32_t)e % BX, g.nx - 1);
            const uint32_t y = min(gy * BY + ((uint32_t)e / BX) % BY, g.ny - 1);
            const uint32_t z = min(gz * BZ + (uint32_t)e / (BX * BY), g.nz - 1);
            qp[e] = (uint32_t)quantize(__ldg(a + (size_t)x + (size_t)g.nx * (y + (size_t)g.ny * z)), r);
        }
        first = (int32_t)qp[0];
#pragma unroll
        for (int e = 31; e >= 0; e--) qp[e] -= qp[0];
        uint32_t mx0 = 0, mx1 = 0;
#pragma unroll
        for (int e = 0; e < 32; e++) {
            const uint32_t dc = e ? qp[e] - qp[e - 1] : 0u;
            const uint32_t ac = (int32_t)dc < 0 ? 0u - dc : dc;
            mx0 = max(mx0, ac);
        }
#pragma unroll
        for (int e = 0; e < 32; e++) {
            const uint32_t ex = (uint32_t)e % BX, ey = ((uint32_t)e / BX) % BY, ez = (uint32_t)e / (BX * BY);
            uint32_t du = 0;
#pragma unroll
            for (uint32_t sm = 0; sm < 8; sm++) {
                const uint32_t sx = sm & 1u, sy = (sm >> 1) & 1u, sz = (sm >> 2) & 1u;
                if (sx > ex || sy > ey || sz > ez) continue;
                const uint32_t v = qp[(ex - sx) + BX * ((ey - sy) + BY * (ez - sz))];
                du = (sx + sy + sz) & 1u ? du - v : du + v;
            }
            mag[e] = du;   // the Lorenzo residual, signed, for now
            const uint32_t al = (int32_t)du < 0 ? 0u - du : du;
            mx1 = max(mx1, al);
        }
        sel = mx1 < mx0 ? 1u : 0u;
        const uint32_t mx = sel ? mx1 : mx0;
        w = 32u - __clz(mx);
#pragma unroll
        for (int e = 0; e < 32; e++) {
            const uint32_t d = sel ? mag[e] : (e ? qp[e] - qp[e - 1] : 0u);
            const bool neg = (int32_t)d < 0;
            if (neg) sgn |= 1u << e;
            mag[e] = neg ? 0u - d : d;
        }
    }
    const uint32_t W = __reduce_max_sync(FULL, w);
    const uint32_t words = (b < nbf && w) ? 1u + w : 0u;
    uint32_t iw = words;
#pragma unroll
    for (int of = 1; of < 32; of <<= 1) {
        const uint32_t a0 = __shfl_up_sync(FULL, iw, of);
        if (lane >= (uint32_t)of) iw += a0;
    }
    if (lane == 31) s_wsum[warp] = iw;
    __syncthreads();
    uint32_t ow = iw - words, tw = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (k < (int)warp) ow += s_wsum[k];
        tw += s_wsum[k];
    }
    if (words) {
        uint32_t* dst = s_buf + ow;
        dst[0] = sgn;
        values_to_planes(W, w, mag, [&](int q, uint32_t pl) { dst[1 + q] = pl; });
    }
    if (b < nbf) {
        o.width[b] = (uint8_t)(w | sel << 7);
        o.first[b] = first;
    }
    {
        const uint32_t cb = __ballot_sync(FULL, b < nbf && w == 0);
        if (lane == 0 && (b >> 5) < (nbf + 31) / 32) o.cbits[b >> 5] = cb;
    }
    if (t == 0) {
        reinterpret_cast<uint32_t*>(tcnt + tile)[0] = tw;
        if (tw) atomicAdd(&c->sl_tile[tile / slice_len(gridDim.x)][0], (unsigned long long)tw);
    }
    __syncthreads();
    uint32_t* slot = o.pay + (size_t)tile * TILE_PAY;
    for (uint32_t k = t; k < tw; k += 256) slot[k] = s_buf[k];
}

// Exclusive prefixes of the tiles' (payload words, extrema) in place, with the
// totals at index ntiles and in the control block.  One CTA, chunks of
// consecutive tiles per thread.
__global__ void __launch_bounds__(1024) k_enc_tile_scan(uint2* tcnt, uint32_t ntiles, Ctrl* c,
                                                        const int* status) {
    griddep_enter();
    __shared__ unsigned long long s_w[33][2];
    if (*status) return;
    unsigned long long tw, tc;
    slice_scan_pairs(
        ntiles, c->sl_tile, [&](uint32_t i) { return tcnt[i]; },
        [&](uint32_t i, unsigned long long pw, unsigned long long pc) {
            tcnt[i] = make_uint2((uint32_t)pw, (uint32_t)pc);
        },
        s_w, tw, tc);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tcnt[ntiles] = make_uint2((uint32_t)tw, (uint32_t)tc);
        c->pay_words = tw;
        c->k_total = tc;
    }
}

// Every tile's payload slot to its place in the payload section (a CTA per
// tile, every thread a few words with all its loads in flight).
__device__ __forceinline__ void copy_slot(const uint32_t* __restrict__ src, uint32_t* dst, uint32_t cnt) {
    for (uint32_t k0 = 0; k0 < cnt; k0 += 4 * 256) {
        uint32_t v[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t k = k0 + j * 256 + threadIdx.x;
            v[j] = k < cnt ? __ldcs(src + k) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t k = k0 + j * 256 + threadIdx.x;
            if (k < cnt) dst[k] = v[j];
        }
    }
}

__global__ void __launch_bounds__(256) k_enc_copy(const uint32_t* __restrict__ scratch, const uint2* tpre,
                                                  uint32_t ntiles, uint32_t* pay, const int* status) {
    griddep_enter();
    if (*status) return;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t p0 = tpre[t].x, cnt = tpre[t + 1].x - p0;
        copy_slot(scratch + (size_t)t * TILE_PAY, pay + p0, cnt);
    }
}

// Rank-sequence encoder: the same codec on the delta sequence (Section IV-A:
// B + LZ and BE again, no QZ), organised like the field encoder: 8192-delta
// tiles, one block per thread, payload to per-tile scratch slots, then a tile
// scan (k_rank_tile_scan) and a copy (k_rank_copy).  The sequence length and
// the section offsets are read from the control block, so the launches do not
// depend on data-dependent sizes.
__global__ void __launch_bounds__(256, 3) k_encode_ranks(const int32_t* __restrict__ delta, Ctrl* c, uint2* tcnt,
                                                         uint32_t* scratch, uint8_t* out, int* status) {
    griddep_enter();
    __shared__ __align__(16) uint32_t s_buf[ENC_TILE_BLOCKS * ENC_ROW];
    __shared__ uint32_t s_wsum[8];
    if (*status) return;
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t k = c->k_total;
    const uint32_t nbd = (uint32_t)cdiv(k, L);
    const uint32_t ntiles = (nbd + ENC_TILE_BLOCKS - 1) / ENC_TILE_BLOCKS;
    Layout lo;
    make_layout(c->g.n, c->nb_fmt, true, c->pay_words, k, 0, lo);
    uint32_t* cbits = reinterpret_cast<uint32_t*>(out + lo.r1);
    uint8_t* width = out + lo.r2;
    int32_t* first = reinterpret_cast<int32_t*>(out + lo.r4);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t p0 = (uint64_t)tile * (ENC_TILE_BLOCKS * 32);
        const uint64_t left = k - p0;
        const uint32_t np = left < (uint64_t)(ENC_TILE_BLOCKS * 32) ? (uint32_t)left : (uint32_t)(ENC_TILE_BLOCKS * 32);
        for (uint32_t i0 = 0; i0 < np; i0 += 4 * 256) {   // four loads in flight per thread
            uint32_t v4[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t i = i0 + j * 256 + t;
                v4[j] = i < np ? (uint32_t)__ldcs(delta + p0 + i) : 0u;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t i = i0 + j * 256 + t;
                if (i < np) s_buf[(i >> 5) * ENC_ROW + (i & 31)] = v4[j];
            }
        }
        __syncthreads();
        const uint32_t b = tile * ENC_TILE_BLOCKS + t;
        uint32_t m[32];
        uint32_t sgn = 0, orr = 0;
        int32_t f = 0;
        if (b < nbd) {
            const uint32_t* row = s_buf + t * ENC_ROW;
            const uint64_t nv64 = k - (uint64_t)b * 32u;
            const uint32_t nvalid = nv64 < 32 ? (uint32_t)nv64 : 32u;
            int32_t prev = 0;
#pragma unroll
            for (int e = 0; e < 32; e++) {
                int32_t q = (int32_t)row[e];
                if (e > 0 && (uint32_t)e >= nvalid) q = prev;   // the tail block repeats its last value
                const int32_t d = e ? q - prev : 0;
                if (e == 0) f = q;
                if (d < 0) sgn |= 1u << e;
                m[e] = (uint32_t)(d < 0 ? -d : d);
                orr |= m[e];
                prev = q;
            }
        }
        const uint32_t w = 32u - __clz(orr);
        const uint32_t W = __reduce_max_sync(FULL, w);   // the warp's widest block: picks the transpose
        const uint32_t words = (b < nbd && w) ? 1u + w : 0u;
        uint32_t iw = words;
#pragma unroll
        for (int of = 1; of < 32; of <<= 1) {
            const uint32_t a0 = __shfl_up_sync(FULL, iw, of);
            if (lane >= (uint32_t)of) iw += a0;
        }
        if (lane == 31) s_wsum[warp] = iw;
        __syncthreads();   // also: every staged value has been read
        uint32_t ow = iw - words, tw = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint32_t v = s_wsum[q];
            if (q < (int)warp) ow += v;
            tw += v;
        }
        if (t == 0) {
            tcnt[tile] = make_uint2(tw, 0u);
            if (tw) atomicAdd(&c->sl_rank[tile / slice_len(ntiles)][0], (unsigned long long)tw);
        }
        if (words) {
            uint32_t* dst = s_buf + ow;
            dst[0] = sgn;
            values_to_planes(W, w, m, [&](int r, uint32_t pl) { dst[1 + r] = pl; });
        }
        if (b < nbd) {
            width[b] = (uint8_t)w;
            first[b] = f;
        }
        {
            const uint32_t cb = __ballot_sync(FULL, b < nbd && w == 0);
            if (lane == 0 && (b >> 5) < (nbd + 31) / 32) cbits[b >> 5] = cb;
        }
        __syncthreads();
        uint32_t* slot = scratch + (size_t)tile * TILE_PAY;
        for (uint32_t q = t; q < tw; q += 256) slot[q] = s_buf[q];
        __syncthreads();
    }
}

// Tile prefixes of the rank payload (tiles of the delta sequence); sets rank_words.
__global__ void __launch_bounds__(1024) k_rank_tile_scan(uint2* tcnt, Ctrl* c, const int* status) {
    griddep_enter();
    __shared__ unsigned long long s_w[33][2];
    if (*status) return;
    const uint32_t nbd = (uint32_t)cdiv(c->k_total, L);
    const uint32_t ntiles = (nbd + ENC_TILE_BLOCKS - 1) / ENC_TILE_BLOCKS;
    unsigned long long tw, tz;
    slice_scan_pairs(
        ntiles, c->sl_rank, [&](uint32_t i) { return tcnt[i]; },
        [&](uint32_t i, unsigned long long pw, unsigned long long) { tcnt[i] = make_uint2((uint32_t)pw, 0u); },
        s_w, tw, tz);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tcnt[ntiles] = make_uint2((uint32_t)tw, 0u);
        c->rank_words = tw;
    }
}

// Rank payload slots to the rank payload section (a CTA per tile).
__global__ void __launch_bounds__(256) k_rank_copy(const uint32_t* __restrict__ scratch, const uint2* tpre,
                                                   const Ctrl* c, uint8_t* out, const int* status) {
    griddep_enter();
    if (*status) return;
    const uint64_t k = c->k_total;
    const uint32_t nbd = (uint32_t)cdiv(k, L);
    const uint32_t ntiles = (nbd + ENC_TILE_BLOCKS - 1) / ENC_TILE_BLOCKS;
    Layout lo;
    make_layout(c->g.n, c->nb_fmt, true, c->pay_words, k, 0, lo);
    uint32_t* pay = reinterpret_cast<uint32_t*>(out + lo.r5);
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t p0 = tpre[t].x, cnt = tpre[t + 1].x - p0;
        copy_slot(scratch + (size_t)t * TILE_PAY, pay + p0, cnt);
    }
}

// ================================================================ rank sort
//
// LSD radix sort of (key, position) pairs, stable, after the "onesweep"
// scheme: one pass builds the digit histograms of every pass; then every pass
// is a single kernel over tiles of 4096 keys.  A tile ranks its keys per digit
// with warp match masks (stable: keys keep their input order within a digit),
// publishes its per-digit counts, and finds its global offset per digit with a
// decoupled look-back over the earlier tiles.  Both lists (maxima: key =
// ord(v); minima: key = ~ord(v)) are sorted by the same launches (blockIdx.y
// selects the list).
//
// Only the bits that vary are sorted: every key lies in the field's key range
// [ord(vmin), ord(vmax)], so the digits come from key - (the list's smallest
// possible key), whose bit length B is known from the range pass.  B <= 8, 16,
// 27 or 32 bits take 1, 2, 3 or 4 passes of ceil(B / passes) <= 9 bits.

constexpr int OS_WARPS = 16;                       // 512 threads: one per digit in the look-back
constexpr int OS_ITEMS = 8;                        // keys per lane
constexpr int OS_TILE = OS_WARPS * 32 * OS_ITEMS;  // 4096
constexpr int OS_ND = 512;                         // most digits of a pass (9 bits)
constexpr uint32_t OS_AGG = 1u << 30, OS_INC = 2u << 30, OS_MASK = (1u << 30) - 1;

struct SortPlan {
    int passes, bits;
    uint32_t base[2];   // subtracted from the keys of list 0 / 1
};

__device__ __forceinline__ SortPlan sort_plan(const Ctrl* c) {
    SortPlan sp;
    const uint32_t kmax = c->max_key, kmin = ~c->min_inv;   // ord(vmax), ord(vmin)
    const uint32_t span = kmax > kmin ? kmax - kmin : 0u;
    const int B = span ? 32 - __clz(span) : 0;
    sp.passes = B == 0 ? 0 : B <= 8 ? 1 : B <= 16 ? 2 : B <= 27 ? 3 : 4;
    sp.bits = sp.passes ? (B + sp.passes - 1) / sp.passes : 0;
    sp.base[0] = kmin;
    sp.base[1] = ~kmax;
    return sp;
}

// Lanes of the warp whose `bits`-bit digit equals this lane's (a match mask
// built from ballots); lanes with ok == false match nobody and nobody them.
__device__ __forceinline__ uint32_t match_digit(uint32_t d, bool ok, int bits) {
    uint32_t m = __ballot_sync(FULL, ok);
#pragma unroll
    for (int b = 0; b < 9; b++) {
        if (b < bits) {
            const uint32_t v = __ballot_sync(FULL, (d >> b) & 1u);
            m &= ((d >> b) & 1u) ? v : ~v;
        }
    }
    return ok ? m : (1u << (threadIdx.x & 31));
}

__device__ __forceinline__ uint32_t list_count(const Ctrl* c, int list) {
    return list ? c->cnt_min : c->cnt_max;
}

// The digit histograms of every pass of both lists, and zeroed look-back
// descriptors for the tiles the passes will use.  Warps count into four
// shared slices, summed at the end.  Records the pass count for the rank
// kernels (the sorted lists end in the second buffer when it is odd).
__global__ void __launch_bounds__(256) k_os_hist(const uint2* s0, const uint2* s1, Ctrl* c,
                                                 uint32_t* ghist /* [2][4][512] */, uint32_t* desc_a,
                                                 uint32_t* desc_b, uint32_t desc_stride, const int* status) {
    griddep_enter();
    __shared__ uint32_t h[4][4 * OS_ND];
    if (*status || c->rank_bitmap) return;
    const SortPlan sp = sort_plan(c);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) c->sort_passes = (uint32_t)sp.passes;
    if (sp.passes == 0) return;
    const int list = blockIdx.y;
    const uint2* s = list ? s1 : s0;
    const uint32_t k = list_count(c, list);
    const uint32_t base = sp.base[list], mask = (1u << sp.bits) - 1u;
    for (int i = threadIdx.x; i < 4 * 4 * OS_ND; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    uint32_t* hw = h[(threadIdx.x >> 5) & 3];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint32_t key = s[i].x - base;
#pragma unroll
        for (int p = 0; p < 4; p++)
            if (p < sp.passes) atomicAdd(&hw[p * OS_ND + ((key >> (p * sp.bits)) & mask)], 1u);
    }
    __syncthreads();
    const uint32_t nd = 1u << sp.bits;
    for (uint32_t i = threadIdx.x; i < 4 * OS_ND; i += blockDim.x) {
        if ((i >> 9) >= (uint32_t)sp.passes || (i & (OS_ND - 1)) >= nd) continue;
        const uint32_t v = h[0][i] + h[1][i] + h[2][i] + h[3][i];
        if (v) atomicAdd(&ghist[list * 4 * OS_ND + i], v);
    }
    // zero the descriptors of the tiles in use (both alternating buffers)
    const uint32_t words = (uint32_t)cdiv(k, OS_TILE) * nd;
    uint32_t* da = desc_a + (size_t)list * desc_stride;
    uint32_t* db = desc_b + (size_t)list * desc_stride;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) {
        da[i] = 0u;
        db[i] = 0u;
    }
}

// exclusive scan of each digit histogram -> digit bases (a CTA of 512 per row)
__global__ void __launch_bounds__(512) k_os_bases(const Ctrl* c, const uint32_t* ghist, uint32_t* base,
                                                  const int* status) {
    griddep_enter();
    __shared__ uint32_t s_w[16];
    if (*status || c->rank_bitmap) return;
    const int row = blockIdx.x;   // list * 4 + pass
    if ((row & 3) >= (int)c->sort_passes) return;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t v = ghist[row * OS_ND + threadIdx.x];
    uint32_t inc = v;
#pragma unroll
    for (int of = 1; of < 32; of <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, inc, of);
        if (lane >= (uint32_t)of) inc += t;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    uint32_t pre = 0;
    for (uint32_t k = 0; k < warp; k++) pre += s_w[k];
    base[row * OS_ND + threadIdx.x] = pre + inc - v;
}

__global__ void __launch_bounds__(OS_WARPS * 32, 2) k_os_pass(const uint2* s0, const uint2* s1, uint2* d0, uint2* d1,
                                                 const Ctrl* c, const uint32_t* base, uint32_t* desc,
                                                 uint32_t* desc_next, uint32_t desc_stride, uint32_t* tile_ctr,
                                                 int pass, int* status) {
    griddep_enter();
    __shared__ uint32_t s_tile;
    __shared__ uint16_t wcnt[OS_WARPS][OS_ND];
    __shared__ uint32_t gofs[OS_ND];
    if (*status || c->rank_bitmap) return;
    const SortPlan sp = sort_plan(c);
    if (pass >= sp.passes) return;
    const int list = blockIdx.y;
    const uint2* src = list ? s1 : s0;
    uint2* dst = list ? d1 : d0;
    const uint32_t k = list_count(c, list);
    const uint32_t ntiles = (uint32_t)cdiv(k, OS_TILE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int shift = pass * sp.bits;
    const uint32_t nd = 1u << sp.bits, mask = nd - 1u, kb = sp.base[list];
    uint32_t* dsc = desc + (size_t)list * desc_stride;
    const uint32_t lt = lanemask_lt();
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&tile_ctr[list], 1u);
        for (int i = threadIdx.x; i < OS_WARPS * OS_ND; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= ntiles) break;
        // load: warp w owns keys [t*4096 + w*256, +256), lane-striped (coalesced)
        const uint32_t wbase = t * OS_TILE + warp * 32 * OS_ITEMS;
        uint2 e[OS_ITEMS];
        uint32_t dg[OS_ITEMS];
        uint32_t rk[OS_ITEMS];
#pragma unroll
        for (int j = 0; j < OS_ITEMS; j++) {
            const uint32_t p = wbase + j * 32 + lane;
            const bool ok = p < k;
            e[j] = ok ? src[p] : make_uint2(0u, 0u);
            dg[j] = ok ? ((e[j].x - kb) >> shift) & mask : (uint32_t)OS_ND + lane;
        }
        // stable local ranks inside the warp, in (j, lane) order
#pragma unroll
        for (int j = 0; j < OS_ITEMS; j++) {
            const bool ok = dg[j] < (uint32_t)OS_ND;
            const uint32_t peers = match_digit(dg[j], ok, sp.bits);
            const int leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (ok && lane == leader) b = wcnt[warp][dg[j]];
            b = __shfl_sync(FULL, b, leader);
            rk[j] = b + __popc(peers & lt);
            __syncwarp();
            if (ok && lane == leader) wcnt[warp][dg[j]] = (uint16_t)(b + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        // per digit: offsets of the warps, tile count, look-back
        for (uint32_t d = threadIdx.x; d < nd; d += blockDim.x) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < OS_WARPS; w++) {
                const uint32_t v = wcnt[w][d];
                wcnt[w][d] = (uint16_t)run;
                run += v;
            }
            const uint32_t tot = run;
            uint32_t pre = 0;
            volatile uint32_t* vd = dsc;
            if (t == 0) {
                vd[d] = OS_INC | tot;
            } else {
                vd[(size_t)t * nd + d] = OS_AGG | tot;
                long long j = (long long)t - 1;
                uint32_t spins = 0;
                while (j >= 0) {
                    const uint32_t v = vd[(size_t)j * nd + d];
                    if (v & OS_INC) {
                        pre += v & OS_MASK;
                        break;
                    }
                    if (v & OS_AGG) {
                        pre += v & OS_MASK;
                        j--;
                        continue;
                    }
                    if (++spins > SPIN_LIMIT) {
                        set_status(status, ST_TIMEOUT);
                        break;
                    }
                    // another look-back ran out: stop waiting (polled every 64 polls)
                    if ((spins & 63u) == 0u && *(volatile int*)status) break;
                    __nanosleep(32);
                }
                vd[(size_t)t * nd + d] = OS_INC | (pre + tot);
            }
            gofs[d] = base[(list * 4 + pass) * OS_ND + d] + pre;
            // the next pass uses the other buffer: clear this tile's entry there
            desc_next[(size_t)list * desc_stride + (size_t)t * nd + d] = 0u;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < OS_ITEMS; j++) {
            if (dg[j] < (uint32_t)OS_ND) dst[gofs[dg[j]] + wcnt[warp][dg[j]] + rk[j]] = e[j];
        }
        __syncthreads();
    }
}

// ============================================================ dense ranks
//
// After sorting, entries of one list are ordered by key; the bin q(v) is
// monotone in v, so entries of a bin are contiguous.  delta = 1 + number of
// distinct keys before it in its bin: an inclusive segmented count of
// "new value" flags with segments at bin changes.  Carried as (h, c): h = a
// segment starts in the range, c = count since the last segment start.

struct SegCnt {
    uint32_t h, c;
};
__device__ __forceinline__ SegCnt seg_op(SegCnt x, SegCnt y) {
    return SegCnt{x.h | y.h, y.h ? y.c : x.c + y.c};
}

// The flags of entries b .. b + RANK_TILE / 256 - 1 (all < k), with each key
// and its bin read once.
constexpr int RANK_PER = RANK_TILE / 256;
__device__ __forceinline__ void rank_elems(const uint2* s, uint32_t b, uint32_t k, int list, float r,
                                           SegCnt (&el)[RANK_PER]) {
    uint32_t kp = b ? s[b - 1].x : 0u;
    int32_t qp = b ? quantize(key_float(list ? ~kp : kp), r) : 0;
#pragma unroll
    for (int j = 0; j < RANK_PER; j++) {
        if (b + j >= k) {
            el[j] = SegCnt{0, 0};
            continue;
        }
        const uint32_t kk = s[b + j].x;
        const int32_t q = quantize(key_float(list ? ~kk : kk), r);
        if (b + j == 0) {
            el[j] = SegCnt{1, 1};
        } else {
            const bool seg = q != qp;
            el[j] = SegCnt{seg ? 1u : 0u, (seg || kk != kp) ? 1u : 0u};
        }
        kp = kk;
        qp = q;
    }
}

// Inclusive scan of a warp's values in lane order (seg_op is associative, not
// commutative).
__device__ __forceinline__ SegCnt warp_seg_scan(SegCnt x) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t h = __shfl_up_sync(FULL, x.h, o), c = __shfl_up_sync(FULL, x.c, o);
        if (lane >= (uint32_t)o) x = seg_op(SegCnt{h, c}, x);
    }
    return x;
}

// Exclusive scan of the CTA's 256 per-thread values after `pre`; also returns
// the CTA total (after pre).  Uses s_tot[8].
__device__ __forceinline__ SegCnt cta_seg_scan(SegCnt x, SegCnt pre, SegCnt* s_tot, SegCnt& total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const SegCnt incl = warp_seg_scan(x);
    SegCnt ex{__shfl_up_sync(FULL, incl.h, 1), __shfl_up_sync(FULL, incl.c, 1)};
    if (lane == 0) ex = SegCnt{0, 0};
    if (lane == 31) s_tot[warp] = incl;
    __syncthreads();
    SegCnt run = pre;
    for (uint32_t k = 0; k < warp; k++) run = seg_op(run, s_tot[k]);
    total = run;
    for (uint32_t k = warp; k < 8; k++) total = seg_op(total, s_tot[k]);
    __syncthreads();
    return seg_op(run, ex);
}

// pass 1: aggregate per tile of RANK_TILE entries
__global__ void __launch_bounds__(256) k_rank_tiles(const uint2* l0, const uint2* l1, const uint2* t0, const uint2* t1,
                                                    const Ctrl* c,
                                                    uint2* agg, uint32_t agg_stride, int G,
                                                    const int* status) {
    griddep_enter();
    __shared__ SegCnt s_tot[8];
    if (*status || c->rank_bitmap) return;
    const int list = blockIdx.y;
    const bool odd = c->sort_passes & 1u;   // an odd number of passes ends in the second buffer
    const uint2* s = list ? (odd ? t1 : l1) : (odd ? t0 : l0);
    const uint32_t k = list ? c->cnt_min : c->cnt_max;
    const float r = c->r_f;
    const uint32_t ntiles = (uint32_t)cdiv(k, RANK_TILE);
    for (uint32_t t = blockIdx.x; t < ntiles; t += G) {
        const uint32_t b = t * RANK_TILE + threadIdx.x * RANK_PER;
        SegCnt el[RANK_PER];
        rank_elems(s, b, k, list, r, el);
        SegCnt acc{0, 0};
#pragma unroll
        for (int j = 0; j < RANK_PER; j++) acc = seg_op(acc, el[j]);
        SegCnt tot;
        cta_seg_scan(acc, SegCnt{0, 0}, s_tot, tot);
        if (threadIdx.x == 0) agg[(size_t)list * agg_stride + t] = make_uint2(tot.h, tot.c);
    }
}

// pass 2: exclusive scan of tile aggregates (one CTA per list, sequential chunks)
__global__ void __launch_bounds__(256) k_rank_scan(uint2* agg, uint32_t agg_stride, const Ctrl* c,
                                                   const int* status) {
    griddep_enter();
    __shared__ SegCnt sh[256];
    if (*status || c->rank_bitmap) return;
    const int list = blockIdx.x;
    const uint32_t k = list ? c->cnt_min : c->cnt_max;
    const uint32_t ntiles = (uint32_t)cdiv(k, RANK_TILE);
    uint2* a = agg + (size_t)list * agg_stride;
    const uint32_t per = (ntiles + 255) / 256;
    const uint32_t b = threadIdx.x * per, e = min(ntiles, b + per);
    SegCnt acc{0, 0};
    for (uint32_t i = b; i < e; i++) acc = seg_op(acc, SegCnt{a[i].x, a[i].y});
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        SegCnt run{0, 0};
        for (int j = 0; j < 256; j++) {
            SegCnt v = sh[j];
            sh[j] = run;
            run = seg_op(run, v);
        }
    }
    __syncthreads();
    SegCnt run = sh[threadIdx.x];
    for (uint32_t i = b; i < e; i++) {
        SegCnt v{a[i].x, a[i].y};
        a[i] = make_uint2(run.h, run.c);
        run = seg_op(run, v);
    }
}

// pass 3: per tile, scan with the carried prefix and scatter delta[pos]
__global__ void __launch_bounds__(256) k_rank_scatter(const uint2* l0, const uint2* l1, const uint2* t0,
                                                      const uint2* t1, const Ctrl* c,
                                                      const uint2* agg, uint32_t agg_stride, const uint2* tpre,
                                                      int32_t* delta, int G, const int* status) {
    griddep_enter();
    __shared__ SegCnt s_tot[8];
    if (*status || c->rank_bitmap) return;
    const int list = blockIdx.y;
    const bool odd = c->sort_passes & 1u;   // an odd number of passes ends in the second buffer
    const uint2* s = list ? (odd ? t1 : l1) : (odd ? t0 : l0);
    const uint32_t k = list ? c->cnt_min : c->cnt_max;
    const float r = c->r_f;
    const uint32_t ntiles = (uint32_t)cdiv(k, RANK_TILE);
    for (uint32_t t = blockIdx.x; t < ntiles; t += G) {
        const uint32_t b = t * RANK_TILE + threadIdx.x * RANK_PER;
        SegCnt el[RANK_PER];
        rank_elems(s, b, k, list, r, el);
        SegCnt acc{0, 0};
#pragma unroll
        for (int j = 0; j < RANK_PER; j++) acc = seg_op(acc, el[j]);
        const uint2 pre = agg[(size_t)list * agg_stride + t];
        SegCnt tot;
        SegCnt run = cta_seg_scan(acc, SegCnt{pre.x, pre.y}, s_tot, tot);
#pragma unroll
        for (int j = 0; j < RANK_PER; j++) {
            if (b + j < k) {
                run = seg_op(run, el[j]);
                const uint32_t y = s[b + j].y;
                delta[tpre[y >> TILE_POS_BITS].y + (y & ((1u << TILE_POS_BITS) - 1))] = (int32_t)run.c;
            }
        }
        __syncthreads();
    }
}

// ================================================================ finalize

__device__ void zero_bytes(uint8_t* out, uint64_t from, uint64_t to) {
    for (uint64_t i = from; i < to; i++) out[i] = 0;
}

template <class T>
__device__ __forceinline__ void put(uint8_t* h, int off, T v) {
    *reinterpret_cast<T*>(h + off) = v;
}

// Header, zero padding between sections, adaptive RBF parameters and the
// stream size.  Section IV-B(3) picks sigma in [0.5, 1] and k in {3, 5, 7} from
// the data's neighbour variation; here V = sum |d| / (pairs * max(1, qmax -
// qmin)) over the integer codes (exact, order independent).
__global__ void k_finalize(Ctrl* c, uint8_t* out, uint64_t* out_size, int32_t rbf_k_over,
                           float rbf_sigma_over, const int* status) {
    griddep_enter();
    __shared__ float s_g[9];
    __shared__ float s_sigma;
    __shared__ int32_t s_k;
    if (blockIdx.x != 0) return;
    if (*status) {
        if (threadIdx.x == 0) *out_size = 0;
        return;
    }
    if (threadIdx.x == 0) {
        // adaptive RBF parameters
        const float r = c->r_f;
        int64_t qmin = quantize(c->vmin, r), qmax = quantize(c->vmax, r);
        int64_t span = qmax - qmin;
        if (span < 1) span = 1;
        const uint64_t pairs = (uint64_t)c->g.n - c->g.nb;
        const double V = pairs ? __ddiv_rn((double)c->sum_abs, __dmul_rn((double)pairs, (double)span)) : 0.0;
        s_sigma = rbf_sigma_over > 0.0f
                      ? rbf_sigma_over
                      : __double2float_rn(__dadd_rn(0.5, __dmul_rn(0.5, __dsub_rn(1.0, fmin(1.0, __ddiv_rn(V, 0.05))))));
        s_k = rbf_k_over > 0 ? rbf_k_over : (V < 0.002 ? 7 : (V < 0.02 ? 5 : 3));
    }
    __syncthreads();
    if (threadIdx.x < 9) {   // one weight per thread: g(d2) for d2 = 1..9
        const double sg = (double)s_sigma;
        const int d2 = threadIdx.x + 1;
        s_g[threadIdx.x] = __double2float_rn(exp_neg(__ddiv_rn((double)d2, __dmul_rn(__dmul_rn(2.0, sg), sg))));
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const Geo g = c->g;
    const bool topo = !(c->flags & FLAG_NO_TOPO);
    const uint64_t k = topo ? c->k_total : 0;
    Layout lo;
    const uint32_t nbf = c->nb_fmt;   // blocks of the stream's format
    make_layout(g.n, nbf, topo, c->pay_words, k, topo ? c->rank_words : 0, lo);
    // padding
    zero_bytes(out, lo.s1 + 4 * cdiv(nbf, 32), lo.s2);
    zero_bytes(out, lo.s2 + nbf, lo.s4);
    zero_bytes(out, lo.s4 + 4ull * nbf, lo.s6);
    zero_bytes(out, lo.s6 + (topo ? 4 * cdiv(g.n, 16) : 0), lo.s5);
    if (topo) {
        uint64_t nbd = cdiv(k, L);
        zero_bytes(out, lo.s5_end, lo.s7);
        zero_bytes(out, lo.r1 + 4 * cdiv(nbd, 32), lo.r2);
        zero_bytes(out, lo.r2 + nbd, lo.r4);
        zero_bytes(out, lo.r4 + 4 * nbd, lo.r5);
    }
    const float sigma = s_sigma;
    const int32_t kk = s_k;
    const float* gw = s_g;
    // header
    uint8_t* h = out;
    for (int i = 0; i < (int)HDR; i += 4) put<uint32_t>(h, i, 0u);
    put<uint32_t>(h, 0, MAGIC);
    put<uint32_t>(h, 4, (c->flags & FLAG_TILE_BLOCKS) ? VERSION_TILES : VERSION);
    put<uint32_t>(h, 8, (uint32_t)g.ndim);
    put<uint32_t>(h, 12, L);
    put<uint64_t>(h, 16, g.nx);
    put<uint64_t>(h, 24, g.ny);
    put<uint64_t>(h, 32, g.nz);
    put<uint32_t>(h, 40, c->flags & (FLAG_NO_TOPO | FLAG_RBF_SOLVE));
    put<uint32_t>(h, 44, (uint32_t)c->rel);
    put<double>(h, 48, c->eb);
    put<double>(h, 56, c->eps);
    put<float>(h, 64, c->w_f);
    put<float>(h, 68, c->r_f);
    put<float>(h, 72, c->h_f);
    put<uint32_t>(h, 76, (uint32_t)c->const_field);
    put<float>(h, 80, c->vmin);
    put<float>(h, 84, c->vmax);
    put<uint32_t>(h, 88, (uint32_t)kk);
    put<float>(h, 92, sigma);
    put<uint32_t>(h, 96, (uint32_t)c->rs_sweeps);
    put<uint64_t>(h, 104, g.n);
    put<uint64_t>(h, 112, nbf);
    put<uint64_t>(h, 120, topo ? c->cnt_min : 0ull);
    put<uint64_t>(h, 128, topo ? c->cnt_max : 0ull);
    put<uint64_t>(h, 136, topo ? c->k_sad : 0ull);
    put<uint64_t>(h, 144, c->sum_abs);
    put<uint64_t>(h, 152, lo.s1);
    put<uint64_t>(h, 160, lo.s2);
    put<uint64_t>(h, 168, lo.s4);
    put<uint64_t>(h, 176, lo.s6);
    put<uint64_t>(h, 184, lo.s5);
    put<uint64_t>(h, 192, topo ? lo.s7 : lo.end);
    put<uint64_t>(h, 200, lo.end);
    put<uint64_t>(h, 208, c->pay_words);
    put<uint32_t>(h, 216, topo ? (uint32_t)c->rank_words : 0u);
    for (int i = 0; i < 9; i++) put<float>(h, 220 + 4 * i, gw[i]);
    *out_size = lo.end;
}

// ============================================================ host launchers

static bool vec_ok(const float* a, const Geo& g) {
    return g.nx % 4 == 0 && (reinterpret_cast<uintptr_t>(a) & 15u) == 0;
}

void launch_range_cd(const float* a, const Geo& g, Ctrl* c, uint32_t* labels, bool topo, int sms,
                     cudaStream_t st) {
    if (vec_ok(a, g)) {
        const int th = g_tuning.cd_threads;
        const uint32_t per_cta_chunks = (uint32_t)th / 32;   // one 128-point chunk per warp
        uint32_t blocks = hmin<uint32_t>((g.n / 128 + per_cta_chunks - 1) / per_cta_chunks + 1,
                                         (uint32_t)sms * (uint32_t)g_tuning.cd_blocks_per_sm);
        const bool three = g.ndim == 3;
        // column segments: at least 48 warps per SM, else (few, short columns)
        // the chunk kernel below, whose n/128 warps are more (cd_columns = 1
        // keeps the column pass there too)
        const uint32_t ncols = g.nxy / 128, want = (uint32_t)sms * 48u;
        uint32_t zseg = CD_ZSEG;
        if ((uint64_t)ncols * ((g.nz + zseg - 1) / zseg) < want)
            zseg = hmax<uint32_t>(CD_ZSEG_MIN, (uint32_t)(((uint64_t)g.nz * ncols + want - 1) / want));
        const uint32_t work = ncols * ((g.nz + zseg - 1) / zseg);   // warps
        if (topo && three && g.nxy % 128 == 0 && g_tuning.cd_columns >= 0 &&
            (g_tuning.cd_columns > 0 || 2 * work >= want)) {
            // 16 CTAs per SM (four waves of the four that fit at 60 registers):
            // shorter tails than one or two waves
            const uint32_t cb = hmin<uint32_t>((work + 7) / 8, (uint32_t)sms * 16);
            launch_pdl(k_range_cd_col, dim3(cb ? cb : 1), dim3(256), 0, st, a, g, c, labels, zseg);
            return;
        }
        if (topo && three) launch_pdl(k_range_cd_vec<true, false, true, true>, dim3(blocks), dim3(th), 0, st, a, g, c, labels, nullptr);
        else if (topo) launch_pdl(k_range_cd_vec<true, false, true, false>, dim3(blocks), dim3(th), 0, st, a, g, c, labels, nullptr);
        else launch_pdl(k_range_cd_vec<false, false, true, false>, dim3(blocks), dim3(th), 0, st, a, g, c, labels, nullptr);
        return;
    }
    uint32_t nchunks = (g.n + 511) / 512;
    uint32_t blocks = hmin<uint32_t>((nchunks + 7) / 8, (uint32_t)sms * 8);
    if (blocks == 0) blocks = 1;
    if (topo) launch_pdl(k_range_cd<true, false, true>, dim3(blocks), dim3(256), 0, st, a, g, c, labels, nullptr);
    else launch_pdl(k_range_cd<false, false, true>, dim3(blocks), dim3(256), 0, st, a, g, c, labels, nullptr);
}

void launch_critical_points(const float* a, const Geo& g, uint32_t* labels, unsigned long long* counts,
                            int sms, cudaStream_t st) {
    if (vec_ok(a, g)) {
        uint32_t blocks = hmin<uint32_t>((g.n / 128 + 7) / 8 + 1, (uint32_t)sms * 8);
        const bool three = g.ndim == 3;
        if (counts) {
            if (three) launch_pdl(k_range_cd_vec<true, true, false, true>, dim3(blocks), dim3(256), 0, st, a, g, nullptr, labels, counts);
            else launch_pdl(k_range_cd_vec<true, true, false, false>, dim3(blocks), dim3(256), 0, st, a, g, nullptr, labels, counts);
            launch_pdl(k_count_regular, dim3(1), dim3(1), 0, st, g.n, counts);
        } else {
            if (three) launch_pdl(k_range_cd_vec<true, false, false, true>, dim3(blocks), dim3(256), 0, st, a, g, nullptr, labels, nullptr);
            else launch_pdl(k_range_cd_vec<true, false, false, false>, dim3(blocks), dim3(256), 0, st, a, g, nullptr, labels, nullptr);
        }
        return;
    }
    uint32_t nchunks = (g.n + 511) / 512;
    uint32_t blocks = hmin<uint32_t>((nchunks + 7) / 8, (uint32_t)sms * 8);
    if (blocks == 0) blocks = 1;
    if (counts) {
        launch_pdl(k_range_cd<true, true, false>, dim3(blocks), dim3(256), 0, st, a, g, nullptr, labels, counts);
        launch_pdl(k_count_regular, dim3(1), dim3(1), 0, st, g.n, counts);
    } else {
        launch_pdl(k_range_cd<true, false, false>, dim3(blocks), dim3(256), 0, st, a, g, nullptr, labels, nullptr);
    }
}

// Section III-B error classes between two packed label maps.
__global__ void k_topo_errors(const uint32_t* a, const uint32_t* b, uint64_t n, unsigned long long* out) {
    griddep_enter();
    __shared__ unsigned long long sh[12];
    if (threadIdx.x < 12) sh[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t nwords = (n + 15) / 16;
    unsigned long long loc[12];
    for (int i = 0; i < 12; i++) loc[i] = 0;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t x = a[w], y = b[w];
        uint32_t diff = x ^ y;
        while (diff) {
            int bit = (__ffs(diff) - 1) & ~1;
            diff &= ~(3u << bit);
            int ta = (x >> bit) & 3, tb = (y >> bit) & 3;
            if (tb == LAB_R) loc[0 * 4 + ta]++;
            else if (ta == LAB_R) loc[1 * 4 + tb]++;
            else loc[2 * 4 + ta]++;
        }
    }
    for (int i = 0; i < 12; i++)
        if (loc[i]) atomicAdd(&sh[i], loc[i]);
    __syncthreads();
    if (threadIdx.x < 12 && sh[threadIdx.x]) atomicAdd(&out[threadIdx.x], sh[threadIdx.x]);
}

void launch_topo_errors(const uint32_t* a, const uint32_t* b, uint64_t n, unsigned long long* out12, int sms,
                        cudaStream_t st) {
    uint64_t nwords = (n + 15) / 16;
    uint32_t blocks = (uint32_t)hmin<uint64_t>((nwords + 255) / 256, (uint64_t)sms * 4);
    if (blocks == 0) blocks = 1;
    launch_pdl(k_topo_errors, dim3(blocks), dim3(256), 0, st, a, b, n, out12);
}

void launch_qparams(Ctrl* c, int* status, cudaStream_t st) { launch_pdl(k_qparams, dim3(1), dim3(32), 0, st, c, status); }

__global__ void __launch_bounds__(256) k_bm_zero(Ctrl* c, uint32_t* region, unsigned long long region_bytes,
                                                 unsigned long long slot_bytes, int mode, const int* status);

void launch_encode_field(const float* a, const uint32_t* labels, Ctrl* c, uint2* tcnt, uint32_t* scratch,
                         uint64_t region_bytes, uint8_t* out, const Layout& lo, uint2* listM, uint2* listm, bool topo,
                         const Geo& g, uint32_t nb_fmt, bool tiles, int sms, int* status, cudaStream_t st) {
    EncOut o{reinterpret_cast<uint32_t*>(out + lo.s1), out + lo.s2,
             reinterpret_cast<int32_t*>(out + lo.s4), scratch};
    // one tile per CTA: the linear 8192-point tiles, or in format v2 as many
    // as either the linear tiles or the payload tiles need
    const uint32_t ntiles = hmax<uint32_t>((g.nb + ENC_TILE_BLOCKS - 1) / ENC_TILE_BLOCKS,
                                           (nb_fmt + ENC_TILE_BLOCKS - 1) / ENC_TILE_BLOCKS);
    if (topo) {
        // the rank mode (key bitmaps or sort) is decided here, so the encoder can set the bits
        const unsigned long long slot_bytes = 4ull * TILE_PAY * ntiles;
        launch_pdl(k_bm_zero, dim3((uint32_t)sms * 8), dim3(256), 0, st, c, scratch, region_bytes, slot_bytes, g_tuning.rank_bitmap,
                                                      status);
        if (tiles) launch_pdl(k_encode_field<true, false>, dim3(ntiles), dim3(256), 0, st, a, labels, c, tcnt, o, listM, listm, scratch, status);
        else launch_pdl(k_encode_field<true, true>, dim3(ntiles), dim3(256), 0, st, a, labels, c, tcnt, o, listM, listm, scratch, status);
    } else {
        if (tiles) launch_pdl(k_encode_field<false, false>, dim3(ntiles), dim3(256), 0, st, a, labels, c, tcnt, o, listM, listm, scratch, status);
        else launch_pdl(k_encode_field<false, true>, dim3(ntiles), dim3(256), 0, st, a, labels, c, tcnt, o, listM, listm, scratch, status);
    }
    if (tiles) {
        if (g.ndim == 3) launch_pdl(k_encode_tiles<3>, dim3(ntiles), dim3(256), 0, st, a, c, tcnt, o, status);
        else launch_pdl(k_encode_tiles<2>, dim3(ntiles), dim3(256), 0, st, a, c, tcnt, o, status);
    }
    launch_pdl(k_enc_tile_scan, dim3(SCAN_SLICES), dim3(1024), 0, st, tcnt, ntiles, c, status);
    uint32_t cg = hmin<uint32_t>(ntiles, (uint32_t)sms * 8);
    launch_pdl(k_enc_copy, dim3(cg ? cg : 1), dim3(256), 0, st, scratch, tcnt, ntiles, reinterpret_cast<uint32_t*>(out + lo.s5),
                                            status);
}

// ====================================================== dense ranks from bitmaps
//
// When the keys' span 2^B (bits of key - smallest key, from the range pass)
// fits the workspace, the dense ranks need no sort.  Per list, a bitmap over
// the span marks the keys present; an exclusive popcount prefix per word gives
// P(x) = number of distinct keys below x.  Bins (QZ codes) are contiguous key
// intervals (quantisation is monotone in the value, ord() in the key), so
// delta = 1 + P(key) - P(lo), lo = the smallest key of the entry's bin.
// Layout at the end of the region (W words, a multiple of 4): bitmap 0,
// bitmap 1, then per list W pairs (prefix, bitmap word), so that P(x) takes one
// 8-byte load.  P(lo) comes from a table over the bins of the field's range
// (the region's start, free once the field payload is copied out) when it
// fits; otherwise each entry finds lo itself.  Same deltas as the sort path.

constexpr uint32_t BM_CHUNK = 8192;   // words per prefix chunk (one CTA)

__device__ __forceinline__ int32_t key_bin(uint32_t key, int list, float r) {
    return quantize(key_float(list ? ~key : key), r);
}

// Decides the mode, sizes the bin table and zeroes the two bitmaps.  The
// bitmaps and pairs take the end of the region (the field encoder's payload
// slots use its start while it sets the bits); c->bm_off is their word offset.
// mode: < 0 the sort, 0 bitmaps and bin table when they fit, 1 no bin table.
__global__ void __launch_bounds__(256) k_bm_zero(Ctrl* c, uint32_t* region, unsigned long long region_bytes,
                                                 unsigned long long slot_bytes, int mode, const int* status) {
    griddep_enter();
    if (*status) return;
    const SortPlan sp = sort_plan(c);
    const uint32_t kmax = c->max_key, kmin = ~c->min_inv;
    const uint32_t span = kmax > kmin ? kmax - kmin : 0u;
    const int B = span ? 32 - __clz(span) : 0;
    const unsigned long long W = B <= 31 ? (((1ull << B) + 31) / 32 + 1 + 3) & ~3ull : 0ull;
    const bool use = mode >= 0 && sp.passes > 0 && B <= 31 && slot_bytes + 24ull * W + 16 <= region_bytes;
    const unsigned long long off = use ? ((region_bytes - 24ull * W) / 4) & ~3ull : 0ull;
    // QZ bins of the range [vmin, vmax]: both lists' entries fall inside
    const float r = c->r_f;
    const long long q0 = quantize(key_float(kmin), r), q1 = quantize(key_float(kmax), r);
    const long long nbins = q1 - q0 + 1;
    const bool tab = use && mode == 0 && nbins > 0 && 8ull * (unsigned long long)nbins <= slot_bytes;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->rank_bitmap = use ? 1u : 0u;
        c->bm_words = use ? (uint32_t)W : 0u;
        c->bm_off = (uint32_t)off;
        c->bin_n = tab ? (uint32_t)nbins : 0u;
        c->bin_q0 = (int32_t)q0;
    }
    if (!use) return;
    uint32_t* bm = region + off;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < 2 * W;
         i += (unsigned long long)gridDim.x * blockDim.x)
        bm[i] = 0u;
}

// popcount of every BM_CHUNK-word chunk of both bitmaps
__global__ void __launch_bounds__(256) k_bm_sums(Ctrl* c, const uint32_t* region, uint32_t* csum,
                                                 const int* status) {
    griddep_enter();
    __shared__ uint32_t s_w[8];
    if (*status || !c->rank_bitmap) return;
    const uint32_t W = c->bm_words, nch = (W + BM_CHUNK - 1) / BM_CHUNK;
    region += c->bm_off;
    for (uint32_t q = blockIdx.x; q < 2 * nch; q += gridDim.x) {
        const uint32_t list = q / nch, ch = q % nch;
        const uint32_t* bm = region + (size_t)list * W + (size_t)ch * BM_CHUNK;
        const uint32_t nw = min(BM_CHUNK, W - ch * BM_CHUNK);   // a multiple of 4, like W
        const uint4* b4 = reinterpret_cast<const uint4*>(bm);
        uint32_t a = 0;
        for (uint32_t i = threadIdx.x; i < nw / 4; i += blockDim.x) {
            const uint4 v = b4[i];
            a += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
        a = __reduce_add_sync(FULL, a);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < 8; w++) t += s_w[w];
            csum[q] = t;
        }
        __syncthreads();
    }
}

// (exclusive popcount prefix, word) of every bitmap word.  A CTA per chunk of
// BM_CHUNK words: 8 consecutive words per thread (16-byte loads and stores;
// W, the region offset and every chunk are 16-byte aligned), a shuffle scan
// per warp, one barrier for the warp totals; the chunk's offset is the sum of
// the chunk sums (csum) before it.
__global__ void __launch_bounds__(1024) k_bm_prefix(Ctrl* c, uint32_t* region, const uint32_t* csum,
                                                    const int* status) {
    griddep_enter();
    __shared__ uint32_t s_o[32], s_wt[32];
    if (*status || !c->rank_bitmap) return;
    const uint32_t W = c->bm_words, nch = (W + BM_CHUNK - 1) / BM_CHUNK;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    region += c->bm_off;
    static_assert(BM_CHUNK == 1024 * 8, "one pass of 8 words per thread");
    for (uint32_t q = blockIdx.x; q < 2 * nch; q += gridDim.x) {
        const uint32_t list = q / nch, ch = q % nch;
        uint32_t o = 0;
        for (uint32_t i = threadIdx.x; i < ch; i += blockDim.x) o += csum[list * nch + i];
        o = __reduce_add_sync(FULL, o);
        if (lane == 0) s_o[warp] = o;
        const uint32_t* bm = region + (size_t)list * W + (size_t)ch * BM_CHUNK;
        uint2* pr = reinterpret_cast<uint2*>(region + 2 * (size_t)W) + (size_t)list * W + (size_t)ch * BM_CHUNK;
        const uint32_t nw = min(BM_CHUNK, W - ch * BM_CHUNK);
        const uint32_t i0 = threadIdx.x * 8;
        const bool full = i0 + 8 <= nw;
        uint32_t w[8];
        if (full) {
            const uint4 x = *reinterpret_cast<const uint4*>(bm + i0);
            const uint4 y = *reinterpret_cast<const uint4*>(bm + i0 + 4);
            w[0] = x.x, w[1] = x.y, w[2] = x.z, w[3] = x.w, w[4] = y.x, w[5] = y.y, w[6] = y.z, w[7] = y.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++) w[j] = i0 + j < nw ? bm[i0 + j] : 0u;
        }
        uint32_t pre[8], run = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            pre[j] = run;
            run += __popc(w[j]);
        }
        uint32_t incl = run;
#pragma unroll
        for (int of = 1; of < 32; of <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, of);
            if (lane >= (uint32_t)of) incl += t;
        }
        if (lane == 31) s_wt[warp] = incl;
        __syncthreads();
        uint32_t base = incl - run;
#pragma unroll
        for (int k = 0; k < 32; k++) {
            base += s_o[k];
            if (k < (int)warp) base += s_wt[k];
        }
        if (full) {
            uint4* d = reinterpret_cast<uint4*>(pr + i0);
#pragma unroll
            for (int j = 0; j < 4; j++)
                d[j] = make_uint4(base + pre[2 * j], w[2 * j], base + pre[2 * j + 1], w[2 * j + 1]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (i0 + j < nw) pr[i0 + j] = make_uint2(base + pre[j], w[j]);
        }
        __syncthreads();   // s_o and s_wt are reused by the next chunk
    }
}

// P(x): distinct keys of the list below relative key x
__device__ __forceinline__ uint32_t bm_below(const uint2* pr, uint32_t x) {
    const uint2 p = pr[x >> 5];
    return p.x + __popc(p.y & ((1u << (x & 31)) - 1u));
}

// Smallest relative key x in [0, hi] whose bin is not before q in the list's
// key order (hi + 1 if none): start from the bin edge (q -+ 0.5) * w in
// binary32, a few ulps off at most, and step to the exact edge; a binary
// search if the steps do not settle.  For a key of bin q and hi = its relative
// key this is the smallest relative key of that bin.
__device__ __forceinline__ uint32_t bin_first(int32_t q, uint32_t hi, uint32_t base, int list, float r, float w_f) {
    auto before = [&](uint32_t x) {
        const int32_t qx = key_bin(x + base, list, r);
        return list ? qx > q : qx < q;
    };
    const float edge = __fmul_rn(list ? (float)q + 0.5f : (float)q - 0.5f, w_f);
    const uint32_t gk = list ? ~ord_key(edge) : ord_key(edge);
    const long long gr = (long long)gk - (long long)base;
    uint32_t x = gr < 0 ? 0u : (gr > (long long)hi ? hi : (uint32_t)gr);
    for (int it = 0; it < 16; it++) {
        if (before(x)) {
            if (x == hi) return hi + 1;
            x++;
        } else if (x > 0 && !before(x - 1)) {
            x--;
        } else {
            return x;
        }
    }
    uint32_t a = 0, b = hi + 1;
    while (a < b) {
        const uint32_t mid = a + ((b - a) >> 1);
        if (before(mid)) a = mid + 1;
        else b = mid;
    }
    return a;
}

// P(lo) of every bin of the field's range, both lists: table[list * bin_n + q - bin_q0]
__global__ void __launch_bounds__(256) k_bin_table(Ctrl* c, uint32_t* region, const int* status) {
    griddep_enter();
    if (*status || !c->rank_bitmap || !c->bin_n) return;
    const SortPlan sp = sort_plan(c);
    const uint32_t W = c->bm_words, nb = c->bin_n;
    const uint32_t span = c->max_key - ~c->min_inv;
    const float r = c->r_f, w_f = c->w_f;
    const uint2* pr0 = reinterpret_cast<const uint2*>(region + c->bm_off + 2 * (size_t)W);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * nb; i += gridDim.x * blockDim.x) {
        const int list = i >= nb;
        const int32_t q = c->bin_q0 + (int32_t)(i - (list ? nb : 0u));
        const uint32_t lo = bin_first(q, span, sp.base[list], list, r, w_f);
        region[i] = bm_below(pr0 + (size_t)list * W, lo);
    }
}

// delta of every list entry; four entries per thread at a time, their table
// lookups in flight together
__global__ void __launch_bounds__(256) k_rank_delta(const uint2* s0, const uint2* s1, Ctrl* c,
                                                    const uint32_t* region, const uint2* tpre, int32_t* delta,
                                                    const int* status) {
    griddep_enter();
    if (*status || !c->rank_bitmap) return;
    const SortPlan sp = sort_plan(c);
    const uint32_t W = c->bm_words, nb = c->bin_n;
    const int32_t q0 = c->bin_q0;
    const float r = c->r_f, w_f = c->w_f;
    const int list = blockIdx.y;
    const uint2* s = list ? s1 : s0;
    const uint32_t k = list_count(c, list), base = sp.base[list];
    const uint2* pr = reinterpret_cast<const uint2*>(region + c->bm_off + 2 * (size_t)W) + (size_t)list * W;
    const uint32_t* tab = region + (size_t)list * nb;
    const uint32_t stride = gridDim.x * blockDim.x;
    constexpr uint32_t TMASK = (1u << TILE_POS_BITS) - 1;
    for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < k; i0 += 4 * stride) {
        uint2 e[4];
        uint32_t rel[4], blo[4], bk[4], tp[4];
#pragma unroll
        for (int j = 0; j < 4; j++) e[j] = i0 + j * stride < k ? s[i0 + j * stride] : make_uint2(base, 0u);
        if (nb) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                rel[j] = e[j].x - base;
                const int32_t q = key_bin(e[j].x, list, r);
                blo[j] = tab[min((uint32_t)(q - q0), nb - 1)];
                bk[j] = bm_below(pr, rel[j]);
                tp[j] = tpre[e[j].y >> TILE_POS_BITS].y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                rel[j] = e[j].x - base;
                const uint32_t lo = bin_first(key_bin(e[j].x, list, r), rel[j], base, list, r, w_f);
                blo[j] = bm_below(pr, lo);
                bk[j] = bm_below(pr, rel[j]);
                tp[j] = tpre[e[j].y >> TILE_POS_BITS].y;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (i0 + j * stride < k) delta[tp[j] + (e[j].y & TMASK)] = (int32_t)(1u + bk[j] - blo[j]);
    }
}

void launch_ranks(Ctrl* c, uint2* listM, uint2* listm, uint2* tmpM, uint2* tmpm, uint64_t tmp_bytes,
                  const SortWs& sw, uint2* agg, uint32_t agg_stride, const uint2* tpre, int32_t* delta, int G,
                  int sms, int* status, cudaStream_t st) {
    // dense ranks from key bitmaps when the key span fits tmpM..tmpm; every
    // kernel of the other path then returns at once (and the other way round)
    (void)tmp_bytes;   // the mode and the bitmaps were set up with the field encoder
    uint32_t* region = reinterpret_cast<uint32_t*>(tmpM);
    uint32_t* csum = reinterpret_cast<uint32_t*>(agg);
    const uint32_t bg = (uint32_t)sms * 8;
    launch_pdl(k_bm_sums, dim3(bg), dim3(256), 0, st, c, region, csum, status);
    launch_pdl(k_bm_prefix, dim3((uint32_t)sms * 2), dim3(1024), 0, st, c, region, csum, status);
    launch_pdl(k_bin_table, dim3((uint32_t)sms * 2), dim3(256), 0, st, c, region, status);
    launch_pdl(k_rank_delta, dim3(bg, 2), dim3(256), 0, st, listM, listm, c, region, tpre, delta, status);
    const uint32_t max_tiles = sw.max_tiles;
    uint32_t hg = hmin<uint32_t>((uint32_t)cdiv((uint64_t)max_tiles * OS_TILE, 256), (uint32_t)sms * 4);
    if (hg == 0) hg = 1;
    launch_pdl(k_os_hist, dim3(hg, 2), dim3(256), 0, st, listM, listm, c, sw.hist, sw.desc_a, sw.desc_b, sw.stride, status);
    launch_pdl(k_os_bases, dim3(8), dim3(OS_ND), 0, st, c, sw.hist, sw.base, status);
    uint2 *a0 = listM, *a1 = listm, *b0 = tmpM, *b1 = tmpm;
    const uint32_t pg = hmin<uint32_t>(max_tiles, (uint32_t)sms * 4);
    for (int pass = 0; pass < 4; pass++) {
        uint32_t* cur = (pass & 1) ? sw.desc_b : sw.desc_a;
        uint32_t* nxt = (pass & 1) ? sw.desc_a : sw.desc_b;
        launch_pdl(k_os_pass, dim3(pg ? pg : 1, 2), dim3(OS_WARPS * 32), 0, st, a0, a1, b0, b1, c, sw.base, cur, nxt, sw.stride,
                                                         sw.ctr + 2 * pass, pass, status);
        uint2* t0 = a0; a0 = b0; b0 = t0;
        uint2* t1 = a1; a1 = b1; b1 = t1;
    }
    // the sorted lists are in listM / listm after an even number of passes,
    // in tmpM / tmpm after an odd one (the kernels read the count)
    dim3 grid(G, 2);
    launch_pdl(k_rank_tiles, dim3(grid), dim3(256), 0, st, listM, listm, tmpM, tmpm, c, agg, agg_stride, G, status);
    launch_pdl(k_rank_scan, dim3(2), dim3(256), 0, st, agg, agg_stride, c, status);
    launch_pdl(k_rank_scatter, dim3(grid), dim3(256), 0, st, listM, listm, tmpM, tmpm, c, agg, agg_stride, tpre, delta, G, status);
}

void launch_encode_ranks(const int32_t* delta, Ctrl* c, uint2* tcnt, uint32_t* scratch, uint8_t* out,
                         uint64_t max_k, int sms, int* status, cudaStream_t st) {
    const uint32_t max_tiles = (uint32_t)cdiv(cdiv(max_k, L), ENC_TILE_BLOCKS);
    uint32_t grid = hmin<uint32_t>(max_tiles, (uint32_t)sms * 3);
    if (grid == 0) grid = 1;
    launch_pdl(k_encode_ranks, dim3(grid), dim3(256), 0, st, delta, c, tcnt, scratch, out, status);
    launch_pdl(k_rank_tile_scan, dim3(SCAN_SLICES), dim3(1024), 0, st, tcnt, c, status);
    uint32_t cg = hmin<uint32_t>(max_tiles, (uint32_t)sms * 8);
    launch_pdl(k_rank_copy, dim3(cg ? cg : 1), dim3(256), 0, st, scratch, tcnt, c, out, status);
}

void launch_finalize(Ctrl* c, uint8_t* out, uint64_t* out_size, int32_t rbf_k, float rbf_sigma,
                     int* status, cudaStream_t st) {
    launch_pdl(k_finalize, dim3(1), dim3(32), 0, st, c, out, out_size, rbf_k, rbf_sigma, status);
}

}  // namespace tsz
