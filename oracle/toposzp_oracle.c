/* TopoSZp CPU oracle -- TEST INFRASTRUCTURE ONLY (see toposzp_oracle.h).
 *
 * Plain single-threaded C11, built with -O2 -ffp-contract=off -fno-fast-math so
 * every float operation below is one IEEE-754 binary32/binary64 operation,
 * rounded to nearest, with no fused multiply-add.  Written from the paper's
 * text; where the paper is silent or garbled the reading taken is stated at the
 * spot, labelled with an R-number.
 */
#include "toposzp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define L 32u                      /* block length (B stage), Section II-C / IV-A */
#define HDR 256u                   /* stream header bytes */
#define MAGIC 0x505A5354u          /* "TSZP" little-endian */
#define VERSION 1u                 /* blocks of L consecutive points (R6) */
#define VERSION_TILES 2u           /* format v2: tile-shaped blocks (R19) */
#define FLAG_NO_TOPO 1u
#define FLAG_RBF_SOLVE 2u
#define FLAG_TILE_BLOCKS 4u        /* compress only: write format v2 */

/* ------------------------------------------------------------------ helpers */

static uint64_t align16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }
static uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

static void put32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
static void put64(uint8_t* p, uint64_t v) { memcpy(p, &v, 8); }
static void putf64(uint8_t* p, double v) { memcpy(p, &v, 8); }
static uint32_t get32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }
static uint64_t get64(const uint8_t* p) { uint64_t v; memcpy(&v, p, 8); return v; }
static double getf64(const uint8_t* p) { double v; memcpy(&v, p, 8); return v; }

/* largest binary32 value <= x (x finite, positive) */
static float f32_round_down(double x) {
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

/* ---------------------------------------------------------- QZ / QZ^ (II-C) */

/* Quantiser constants.  The paper's bin index q = floor((a+eps)/(2 eps)) is the
 * round-half-up of a/(2 eps), and its decode maps q to the bin centre 2 eps q
 * (the printed "q(2eps) - eps" is the bin's lower edge and would break the
 * stated |a - a^| <= eps, reading R4).  In binary32 the products round, so the
 * half-width is shrunk to h = eps - (M + eps) 2^-21 with M = max|a| (R3); then
 * |a - a^| <= h + 4 M 2^-24 + 3 eps 2^-24 < eps for every representable input. */
int orc_qparams_compute(const float* a, uint64_t n, int rel, double eb, orc_qparams* p) {
    memset(p, 0, sizeof(*p));
    float vmin = a[0], vmax = a[0];
    for (uint64_t i = 0; i < n; i++) {
        float v = a[i];
        if (!isfinite(v)) return ORC_NONFINITE;
        if (v < vmin) vmin = v;
        if (v > vmax) vmax = v;
    }
    /* -0 and +0 compare equal; store the range with +0 so its bits are unique */
    if (vmin == 0.0f) vmin = 0.0f;
    if (vmax == 0.0f) vmax = 0.0f;
    p->vmin = vmin;
    p->vmax = vmax;
    double eps = rel ? eb * ((double)vmax - (double)vmin) : eb;
    p->eps = eps;
    if (vmax == vmin) {
        /* constant field: pick the bin width so the constant is reproduced
         * exactly (q = +-1 or 0); no critical points exist. */
        float w = (vmin == 0.0f) ? 1.0f : fabsf(vmin);
        p->const_field = 1;
        p->w_f = w;
        p->r_f = (float)(1.0 / (double)w);
        p->h_f = 0.0f;
        return ORC_OK;
    }
    if (!(eps > 0.0) || !isfinite(eps)) return ORC_EB_TOO_SMALL;
    double M = fmax(fabs((double)vmin), fabs((double)vmax));
    double h = eps - (M + eps) * 0x1p-21;
    if (!(h >= eps * 0.5)) return ORC_EB_TOO_SMALL;
    if (!(2.0 * h <= (double)3.0e38f)) return ORC_INVALID_ARG;
    p->w_f = f32_round_down(2.0 * h);
    p->r_f = (float)(1.0 / (double)p->w_f);
    p->h_f = f32_round_down(h);
    return ORC_OK;
}

int32_t orc_quantize(float a, const orc_qparams* p) {
    float x = a * p->r_f;          /* one rounded binary32 product */
    float y = x + 0.5f;            /* one rounded binary32 sum */
    return (int32_t)floorf(y);
}

float orc_dequantize(int32_t q, const orc_qparams* p) {
    return (float)q * p->w_f;      /* (float)q is exact: |q| <= 2^20 + 1 */
}

/* ------------------------------------------------------- CD (Section IV-A(1)) */

/* Strict comparisons with the face neighbours that lie inside the (non-periodic)
 * grid.  m: every neighbour higher; M: every neighbour lower (so corners use two
 * neighbours and edges three).  s: the point has both neighbours on every axis,
 * each opposite pair is entirely higher (H) or entirely lower (L), and there is
 * at least one H pair and one L pair -- in 2D exactly "t,d higher and l,r lower
 * or vice versa"; in 3D the same rule over three pairs (R9).  Ties are never
 * strict.  A grid of one point has no neighbours and is regular. */
int orc_classify(const float* a, int ndim, const uint64_t dims[3], uint64_t i) {
    uint64_t stride[3] = {1, dims[0], dims[0] * dims[1]};
    uint64_t c[3];
    c[0] = i % dims[0];
    c[1] = (i / dims[0]) % dims[1];
    c[2] = (ndim == 3) ? i / (dims[0] * dims[1]) : 0;
    float v = a[i];
    int nn = 0, nhi = 0, nlo = 0, interior = 1, ph = 0, pl = 0, px = 0;
    for (int ax = 0; ax < ndim; ax++) {
        int has_lo = c[ax] > 0;
        int has_hi = c[ax] + 1 < dims[ax];
        int hc = 0, lc = 0;
        if (has_lo) {
            float u = a[i - stride[ax]];
            nn++;
            if (u > v) { nhi++; hc++; } else if (u < v) { nlo++; lc++; }
        }
        if (has_hi) {
            float u = a[i + stride[ax]];
            nn++;
            if (u > v) { nhi++; hc++; } else if (u < v) { nlo++; lc++; }
        }
        if (has_lo && has_hi) {
            if (hc == 2) ph++;
            else if (lc == 2) pl++;
            else px++;
        } else {
            interior = 0;
        }
    }
    if (nn == 0) return ORC_R;
    if (nhi == nn) return ORC_MIN;
    if (nlo == nn) return ORC_MAX;
    if (interior && px == 0 && ph > 0 && pl > 0) return ORC_SAD;
    return ORC_R;
}

void orc_critical_points(const float* a, int ndim, const uint64_t dims[3], uint8_t* labels) {
    uint64_t n = dims[0] * dims[1] * (ndim == 3 ? dims[2] : 1);
    for (uint64_t i = 0; i < n; i++) labels[i] = (uint8_t)orc_classify(a, ndim, dims, i);
}

/* ------------------------------------------------------- RP (Section IV-A(2)) */

typedef struct { float v; uint64_t idx; } vi_t;

static int cmp_vi_asc(const void* x, const void* y) {
    float a = ((const vi_t*)x)->v, b = ((const vi_t*)y)->v;
    return (a < b) ? -1 : (a > b) ? 1 : 0;
}
static int cmp_vi_desc(const void* x, const void* y) { return -cmp_vi_asc(x, y); }

/* Rank of each extremum among the extrema of its own type in its own
 * quantisation bin (R11): for a maximum, 1 + the number of distinct smaller
 * maximum values in the bin (so M1 < M2 get 1, 2 as in Fig. 5); for a minimum,
 * 1 + the number of distinct larger minimum values in the bin, so that the
 * minimum stencil "min - delta*eta" keeps the original order.  Equal values get
 * equal rank.  Saddles carry no rank (only the extrema stencils use delta).
 * Output: one delta per m/M point, in increasing linear index. */
uint64_t orc_ranks(const float* a, const uint8_t* labels, uint64_t n, const orc_qparams* p,
                   int32_t* delta_seq) {
    uint64_t k = 0;
    for (uint64_t i = 0; i < n; i++) k += (labels[i] == ORC_MIN || labels[i] == ORC_MAX);
    if (k == 0) return 0;
    int32_t* delta_at = (int32_t*)calloc(n, sizeof(int32_t));
    vi_t* list = (vi_t*)malloc(k * sizeof(vi_t));
    for (int type = ORC_MIN; type <= ORC_MAX; type += 2) {
        uint64_t c = 0;
        for (uint64_t i = 0; i < n; i++)
            if (labels[i] == type) { list[c].v = a[i]; list[c].idx = i; c++; }
        qsort(list, c, sizeof(vi_t), type == ORC_MAX ? cmp_vi_asc : cmp_vi_desc);
        int32_t rank = 0;
        for (uint64_t j = 0; j < c; j++) {
            int new_bin = (j == 0) ||
                orc_quantize(list[j].v, p) != orc_quantize(list[j - 1].v, p);
            if (new_bin) rank = 1;
            else if (list[j].v != list[j - 1].v) rank++;
            delta_at[list[j].idx] = rank;
        }
    }
    uint64_t pos = 0;
    for (uint64_t i = 0; i < n; i++)
        if (labels[i] == ORC_MIN || labels[i] == ORC_MAX) delta_seq[pos++] = delta_at[i];
    free(list);
    free(delta_at);
    return k;
}

/* ------------------------------------------------ B + LZ + BE (II-C, IV-A) */

typedef struct {
    uint64_t nblk;
    uint32_t* cbits;   /* (1) constant-block bitmap */
    uint8_t* width;    /* (2) fixed-length block metadata: bit width w_b */
    int32_t* first;    /* (4) first element of each block */
    uint32_t* pay;     /* (3)+(5) per non-constant block: sign plane, w_b planes */
    uint64_t pay_words;
    uint64_t sum_abs;  /* sum of |d| over all blocks (neighbour variation) */
} codec_t;

/* Blocks of L consecutive codes in linear order (R6); the tail block is padded
 * with its last code.  Lorenzo residuals d_0 = 0, d_j = q_j - q_{j-1}.  A block
 * whose residuals are all zero is constant and stores only its first value.
 * Otherwise w_b = bit length of max |d_j|; one sign plane and w_b magnitude
 * planes (plane j holds bit j of |d_i| at bit i) are stored. */
static void codec_encode(const int32_t* q, uint64_t len, codec_t* cd) {
    uint64_t nblk = cdiv(len, L);
    cd->nblk = nblk;
    cd->cbits = (uint32_t*)calloc(cdiv(nblk, 32) + 1, 4);
    cd->width = (uint8_t*)calloc(nblk + 1, 1);
    cd->first = (int32_t*)calloc(nblk + 1, 4);
    cd->pay = (uint32_t*)calloc(nblk * (L + 1) + 1, 4);
    cd->pay_words = 0;
    cd->sum_abs = 0;
    for (uint64_t b = 0; b < nblk; b++) {
        int32_t qq[L];
        uint32_t mag[L];
        int neg[L];
        uint64_t base = b * L;
        for (uint32_t j = 0; j < L; j++) qq[j] = (base + j < len) ? q[base + j] : qq[j - 1];
        uint32_t mx = 0;
        for (uint32_t j = 0; j < L; j++) {
            int64_t d = (j == 0) ? 0 : (int64_t)qq[j] - (int64_t)qq[j - 1];
            neg[j] = d < 0;
            mag[j] = (uint32_t)(d < 0 ? -d : d);
            if (mag[j] > mx) mx = mag[j];
            cd->sum_abs += mag[j];
        }
        uint32_t w = 0;
        while (w < 32 && (mx >> w) != 0) w++;
        cd->width[b] = (uint8_t)w;
        cd->first[b] = qq[0];
        if (w == 0) {
            cd->cbits[b / 32] |= 1u << (b % 32);
            continue;
        }
        uint32_t sgn = 0;
        for (uint32_t j = 0; j < L; j++) sgn |= (uint32_t)neg[j] << j;
        cd->pay[cd->pay_words++] = sgn;
        for (uint32_t pl = 0; pl < w; pl++) {
            uint32_t word = 0;
            for (uint32_t j = 0; j < L; j++) word |= ((mag[j] >> pl) & 1u) << j;
            cd->pay[cd->pay_words++] = word;
        }
    }
}

static void codec_free(codec_t* cd) {
    free(cd->cbits); free(cd->width); free(cd->first); free(cd->pay);
}

/* Inverse: BE^ then LZ^ + B^.  Returns 0 on success, -1 if the payload runs out. */
static int codec_decode(const uint8_t* width, const int32_t* first, const uint32_t* pay,
                        uint64_t pay_words, uint64_t len, int32_t* q) {
    uint64_t nblk = cdiv(len, L), off = 0;
    for (uint64_t b = 0; b < nblk; b++) {
        uint32_t w = width[b];
        int32_t vals[L];
        if (w > 32) return -1;
        if (w == 0) {
            for (uint32_t j = 0; j < L; j++) vals[j] = first[b];
        } else {
            if (off + 1 + w > pay_words) return -1;
            uint32_t sgn = pay[off];
            int64_t acc = first[b];
            for (uint32_t j = 0; j < L; j++) {
                uint32_t m = 0;
                for (uint32_t pl = 0; pl < w; pl++) m |= ((pay[off + 1 + pl] >> j) & 1u) << pl;
                int64_t d = ((sgn >> j) & 1u) ? -(int64_t)m : (int64_t)m;
                if (j > 0) acc += d;
                vals[j] = (int32_t)acc;
            }
            off += 1 + w;
        }
        for (uint32_t j = 0; j < L && b * L + j < len; j++) q[b * L + j] = vals[j];
    }
    return off == pay_words ? 0 : -1;
}

/* Format v2 (R19): tile-shaped blocks of L = 32 points, 8 x 4 in 2D and
 * 4 x 4 x 2 in 3D (x fastest), in raster order over the block grid.  Element
 * e of a block sits at (e mod BX, (e / BX) mod BY, e / (BX BY)) inside it;
 * a position outside the domain takes the code of the nearest point inside
 * (each coordinate clamped).  The residuals are the Lorenzo differences of
 * q' = q - q_0 inside the block, with q' = 0 outside it (the 2D predictor
 * q'(x-1,y) + q'(x,y-1) - q'(x-1,y-1), its 3D analogue over the seven
 * preceding corners), in 32-bit modular arithmetic; the decoder undoes them
 * with prefix sums along x, y and z.  d_0 = 0, and the block's first value
 * q_0, width, sign plane and magnitude planes are stored as in format v1. */
static void tile_shape(int ndim, uint32_t* bx, uint32_t* by, uint32_t* bz) {
    *bx = ndim == 3 ? 4u : 8u;
    *by = 4u;
    *bz = ndim == 3 ? 2u : 1u;
}

uint64_t orc_tile_blocks(int ndim, const uint64_t dims[3]) {
    uint32_t bx, by, bz;
    tile_shape(ndim, &bx, &by, &bz);
    uint64_t nz = ndim == 3 ? dims[2] : 1;
    return cdiv(dims[0], bx) * cdiv(dims[1], by) * cdiv(nz, bz);
}

/* the block's codes q'[e] = q[e] - q[0] of block (gx, gy, gz), e in element order */
static void tile_gather(const int32_t* q, const uint64_t d3[3], uint32_t bx, uint32_t by, uint32_t bz,
                        uint64_t gx, uint64_t gy, uint64_t gz, int32_t qq[L]) {
    for (uint32_t e = 0; e < L; e++) {
        uint64_t x = gx * bx + e % bx, y = gy * by + (e / bx) % by, z = gz * bz + e / (bx * by);
        if (x >= d3[0]) x = d3[0] - 1;
        if (y >= d3[1]) y = d3[1] - 1;
        if (z >= d3[2]) z = d3[2] - 1;
        qq[e] = q[x + d3[0] * (y + d3[1] * z)];
    }
}

static void codec_encode_tiles(const int32_t* q, int ndim, const uint64_t d3[3], codec_t* cd) {
    uint32_t bx, by, bz;
    tile_shape(ndim, &bx, &by, &bz);
    const uint64_t nbx = cdiv(d3[0], bx), nby = cdiv(d3[1], by), nbz = cdiv(d3[2], bz);
    const uint64_t nblk = nbx * nby * nbz;
    cd->nblk = nblk;
    cd->cbits = (uint32_t*)calloc(cdiv(nblk, 32) + 1, 4);
    cd->width = (uint8_t*)calloc(nblk + 1, 1);
    cd->first = (int32_t*)calloc(nblk + 1, 4);
    cd->pay = (uint32_t*)calloc(nblk * (L + 1) + 1, 4);
    cd->pay_words = 0;
    cd->sum_abs = 0;   /* not used by format v2: the linear-block sum is taken */
    for (uint64_t b = 0; b < nblk; b++) {
        int32_t qq[L];
        tile_gather(q, d3, bx, by, bz, b % nbx, (b / nbx) % nby, b / (nbx * nby), qq);
        uint32_t qp[L];   /* q' modulo 2^32 */
        for (uint32_t e = 0; e < L; e++) qp[e] = (uint32_t)qq[e] - (uint32_t)qq[0];
        /* both predictors: 0 = the chain in element order, 1 = Lorenzo */
        uint32_t mag2[2][L], sgn2[2] = {0, 0}, mx2[2] = {0, 0};
        for (uint32_t e = 0; e < L; e++) {
            const uint32_t ex = e % bx, ey = (e / bx) % by, ez = e / (bx * by);
            /* inclusion-exclusion over the corners (ex - sx, ey - sy, ez - sz), s in {0,1}^3 */
            uint32_t du = 0;
            for (uint32_t sm = 0; sm < 8; sm++) {
                const uint32_t sx = sm & 1u, sy = (sm >> 1) & 1u, sz = (sm >> 2) & 1u;
                if (sx > ex || sy > ey || sz > ez) continue;
                const uint32_t v = qp[(ex - sx) + bx * ((ey - sy) + by * (ez - sz))];
                if ((sx + sy + sz) & 1u) du -= v;
                else du += v;
            }
            const uint32_t dc = e ? qp[e] - qp[e - 1] : 0u;
            const uint32_t dd[2] = {dc, du};
            for (int k = 0; k < 2; k++) {
                int32_t d;
                memcpy(&d, &dd[k], 4);
                if (d < 0) sgn2[k] |= 1u << e;
                mag2[k][e] = d < 0 ? (uint32_t)(-(int64_t)d) : (uint32_t)d;
                if (mag2[k][e] > mx2[k]) mx2[k] = mag2[k][e];
            }
        }
        const int sel = mx2[1] < mx2[0];
        const uint32_t* mag = mag2[sel];
        const uint32_t sgn = sgn2[sel], mx = mx2[sel];
        uint32_t w = 0;
        while (w < 32 && (mx >> w) != 0) w++;
        cd->width[b] = (uint8_t)(w | (uint32_t)sel << 7);
        cd->first[b] = qq[0];
        if (w == 0) {
            cd->cbits[b / 32] |= 1u << (b % 32);
            continue;
        }
        cd->pay[cd->pay_words++] = sgn;
        for (uint32_t pl = 0; pl < w; pl++) {
            uint32_t word = 0;
            for (uint32_t e = 0; e < L; e++) word |= ((mag[e] >> pl) & 1u) << e;
            cd->pay[cd->pay_words++] = word;
        }
    }
}

/* Inverse of codec_encode_tiles: residuals, prefix sums along x, then y, then
 * z (modulo 2^32), plus q_0; positions outside the domain are dropped. */
static int codec_decode_tiles(const uint8_t* width, const int32_t* first, const uint32_t* pay, uint64_t pay_words,
                              int ndim, const uint64_t d3[3], int32_t* q) {
    uint32_t bx, by, bz;
    tile_shape(ndim, &bx, &by, &bz);
    const uint64_t nbx = cdiv(d3[0], bx), nby = cdiv(d3[1], by), nbz = cdiv(d3[2], bz);
    const uint64_t nblk = nbx * nby * nbz;
    uint64_t off = 0;
    for (uint64_t b = 0; b < nblk; b++) {
        const uint32_t w = width[b] & 0x7Fu, sel = width[b] >> 7;
        uint32_t acc[L];
        if (w > 32 || (sel && w == 0)) return -1;
        if (w == 0) {
            for (uint32_t e = 0; e < L; e++) acc[e] = 0;
        } else if (!sel) {
            if (off + 1 + w > pay_words) return -1;
            const uint32_t sgn = pay[off];
            for (uint32_t e = 0; e < L; e++) {
                uint32_t m = 0;
                for (uint32_t pl = 0; pl < w; pl++) m |= ((pay[off + 1 + pl] >> e) & 1u) << pl;
                acc[e] = ((sgn >> e) & 1u) ? 0u - m : m;
            }
            off += 1 + w;
            for (uint32_t e = 1; e < L; e++) acc[e] += acc[e - 1];   /* the element-order chain */
        } else {
            if (off + 1 + w > pay_words) return -1;
            const uint32_t sgn = pay[off];
            for (uint32_t e = 0; e < L; e++) {
                uint32_t m = 0;
                for (uint32_t pl = 0; pl < w; pl++) m |= ((pay[off + 1 + pl] >> e) & 1u) << pl;
                acc[e] = ((sgn >> e) & 1u) ? 0u - m : m;
            }
            off += 1 + w;
            for (uint32_t e = 0; e < L; e++)   /* along x */
                if (e % bx) acc[e] += acc[e - 1];
            for (uint32_t e = 0; e < L; e++)   /* along y */
                if ((e / bx) % by) acc[e] += acc[e - bx];
            for (uint32_t e = 0; e < L; e++)   /* along z */
                if (e / (bx * by)) acc[e] += acc[e - bx * by];
        }
        const uint64_t gx = b % nbx, gy = (b / nbx) % nby, gz = b / (nbx * nby);
        for (uint32_t e = 0; e < L; e++) {
            const uint64_t x = gx * bx + e % bx, y = gy * by + (e / bx) % by, z = gz * bz + e / (bx * by);
            if (x >= d3[0] || y >= d3[1] || z >= d3[2]) continue;
            const uint32_t v = acc[e] + (uint32_t)first[b];
            int32_t vi;
            memcpy(&vi, &v, 4);
            q[x + d3[0] * (y + d3[1] * z)] = vi;
        }
    }
    return off == pay_words ? 0 : -1;
}

/* The neighbour variation of the RBF parameters, sum |q_j - q_{j-1}| within
 * blocks of L consecutive points (format v1's residual sum), for either format. */
static uint64_t linear_sum_abs(const int32_t* q, uint64_t n) {
    uint64_t s = 0;
    for (uint64_t i = 1; i < n; i++) {
        if (i % L == 0) continue;
        const int64_t d = (int64_t)q[i] - (int64_t)q[i - 1];
        s += (uint64_t)(d < 0 ? -d : d);
    }
    return s;
}

/* ----------------------------------------------------- RBF parameters (IV-B) */

/* exp(-t) for t >= 0 by scaling and squaring: exp(-t) = (exp(-t/1024))^1024 with
 * a 12-term Taylor polynomial for the small argument.  Only + * / in binary64,
 * so any IEEE machine gives the same bits. */
double orc_exp_neg(double t) {
    double y = -t / 1024.0;
    double e = 1.0;
    for (int j = 12; j >= 1; j--) e = 1.0 + (y / (double)j) * e;
    for (int i = 0; i < 10; i++) e = e * e;
    return e;
}

/* Adaptive sigma in [0.5, 1] and kernel size in {3,5,7} (Section IV-B(3)):
 * driven by the normalised neighbour variation V = sum|d| / (pairs * max(1,
 * q_max - q_min)) of the integer codes, so it is exact and order independent.
 * Smooth data (small V) gets the larger sigma and kernel.  Thresholds are ours. */
static void rbf_params(uint64_t sum_abs, uint64_t n, uint64_t nblk, int32_t qmin, int32_t qmax,
                       int32_t k_over, float s_over, int32_t* k_out, float* s_out, float g[9]) {
    uint64_t pairs = n - nblk;
    int64_t span = (int64_t)qmax - (int64_t)qmin;
    if (span < 1) span = 1;
    double V = pairs ? (double)sum_abs / ((double)pairs * (double)span) : 0.0;
    float sigma = s_over > 0.0f ? s_over : (float)(0.5 + 0.5 * (1.0 - fmin(1.0, V / 0.05)));
    int32_t k = k_over > 0 ? k_over : (V < 0.002 ? 7 : (V < 0.02 ? 5 : 3));
    double s = (double)sigma;
    for (int d2 = 1; d2 <= 9; d2++) g[d2 - 1] = (float)orc_exp_neg((double)d2 / (2.0 * s * s));
    *k_out = k;
    *s_out = sigma;
}

/* Literal RBF interpolation (Section IV-B(3), Eqs. RBF-interp-final and
 * RBF-eval): an interpolant through the values at the nodes q_i of
 * N_r(p) \ {p} (p itself excluded: with p a node, the interpolant would
 * return p's own value), phi(d) = exp(-d^2 / (2 sigma^2)).  Eq. RBF-eval
 * states weights that sum to one; the bare Gaussian interpolant's do not
 * (0.41 - 1.45 over the radii and widths used), so the interpolant carries a
 * constant term, the polynomial-augmented form of RBF interpolation that
 * reproduces constants: s(x) = sum_i w_i phi(|x - q_i|) + c with sum_i w_i = 0.
 * Its value at a point e is alpha^T f with fixed weights alpha for fixed
 * offsets and sigma.  Phi is symmetric positive definite: a Cholesky
 * factorisation L L^T (the textbook order: each entry minus the products of
 * earlier columns, k ascending), forward and back substitution for
 * a = Phi^-1 phi_e and b = Phi^-1 1, and by elimination of c
 *     alpha = a + b (1 - sum a) / sum b        (sums i ascending).
 * Binary64 throughout; exp by orc_exp_neg. */
int orc_rbf_solve(int ndim, int r, float sigma, int ex, int ey, int ez, double* alpha) {
    int ox[343], oy[343], oz[343], m = 0;
    const int rz = ndim == 3 ? r : 0;
    for (int dz = -rz; dz <= rz; dz++)
        for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
                const int d2 = dx * dx + dy * dy + dz * dz;
                if (d2 == 0 || d2 > r * r) continue;
                ox[m] = dx, oy[m] = dy, oz[m] = dz;
                m++;
            }
    const double s = (double)sigma;
    double* Lm = (double*)malloc((size_t)m * m * sizeof(double));
    double* y = (double*)malloc((size_t)m * sizeof(double));
    for (int i = 0; i < m; i++)
        for (int j = 0; j <= i; j++) {
            const int a = ox[i] - ox[j], b = oy[i] - oy[j], c = oz[i] - oz[j];
            Lm[(size_t)i * m + j] = orc_exp_neg((double)(a * a + b * b + c * c) / (2.0 * s * s));
        }
    for (int j = 0; j < m; j++) {
        double d = Lm[(size_t)j * m + j];
        for (int k = 0; k < j; k++) d = d - Lm[(size_t)j * m + k] * Lm[(size_t)j * m + k];
        const double ljj = sqrt(d);
        Lm[(size_t)j * m + j] = ljj;
        for (int i = j + 1; i < m; i++) {
            double t = Lm[(size_t)i * m + j];
            for (int k = 0; k < j; k++) t = t - Lm[(size_t)i * m + k] * Lm[(size_t)j * m + k];
            Lm[(size_t)i * m + j] = t / ljj;
        }
    }
    double* sol[2] = {alpha, (double*)malloc((size_t)m * sizeof(double))};
    for (int rhs = 0; rhs < 2; rhs++) {
        for (int i = 0; i < m; i++) {   /* L y = phi_e, then L y = 1 */
            const int a = ox[i] - ex, b = oy[i] - ey, c = oz[i] - ez;
            double t = rhs == 0 ? orc_exp_neg((double)(a * a + b * b + c * c) / (2.0 * s * s)) : 1.0;
            for (int k = 0; k < i; k++) t = t - Lm[(size_t)i * m + k] * y[k];
            y[i] = t / Lm[(size_t)i * m + i];
        }
        double* x = sol[rhs];
        for (int i = m - 1; i >= 0; i--) {   /* L^T x = y */
            double t = y[i];
            for (int k = m - 1; k > i; k--) t = t - Lm[(size_t)k * m + i] * x[k];
            x[i] = t / Lm[(size_t)i * m + i];
        }
    }
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < m; i++) sa = sa + alpha[i];
    for (int i = 0; i < m; i++) sb = sb + sol[1][i];
    const double cf = (1.0 - sa) / sb;
    for (int i = 0; i < m; i++) alpha[i] = alpha[i] + sol[1][i] * cf;
    free(sol[1]);
    free(Lm);
    free(y);
    return m;
}

/* ------------------------------------------------------------ stream layout */

typedef struct {
    uint64_t s1, s2, s4, s6, s5, s7, end;   /* byte offsets */
} layout_t;

static void field_layout(uint64_t n, uint64_t nblk, int topo, uint64_t pay_words, layout_t* lo) {
    lo->s1 = HDR;
    lo->s2 = align16(lo->s1 + 4 * cdiv(nblk, 32));
    lo->s4 = align16(lo->s2 + nblk);
    lo->s6 = align16(lo->s4 + 4 * nblk);
    lo->s5 = align16(lo->s6 + (topo ? 4 * cdiv(n, 16) : 0));
    lo->s7 = align16(lo->s5 + 4 * pay_words);
    lo->end = lo->s5 + 4 * pay_words;
}

/* nested rank stream (7): its own (1), (2), (4), (3)+(5) sub-sections */
static void rank_layout(uint64_t s7, uint64_t k, uint64_t rpay, uint64_t sub[5]) {
    uint64_t nbd = cdiv(k, L);
    sub[0] = s7;
    sub[1] = align16(sub[0] + 4 * cdiv(nbd, 32));
    sub[2] = align16(sub[1] + nbd);
    sub[3] = align16(sub[2] + 4 * nbd);
    sub[4] = sub[3] + 4 * rpay;          /* end */
}

uint64_t orc_compress_bound(int ndim, const uint64_t dims[3]) {
    uint64_t n = dims[0] * dims[1] * (ndim == 3 ? dims[2] : 1);
    uint64_t nb = cdiv(n, L);
    const uint64_t nbt = orc_tile_blocks(ndim, dims);   /* format v2's block count */
    if (nbt > nb) nb = nbt;
    return HDR + 16 * 12 + 2 * (4 * cdiv(nb, 32) + nb + 4 * nb) + 4 * cdiv(n, 16) +
           4 * (L + 1) * nb + 4 * L * nb;
}

/* ------------------------------------------------------------------ compress */

int orc_compress(const float* a, int ndim, const uint64_t dims[3], int rel, double eb,
                 uint32_t flags, uint32_t rs_sweeps, int32_t rbf_k, float rbf_sigma,
                 uint8_t* out, uint64_t cap, uint64_t* out_size) {
    if (ndim != 2 && ndim != 3) return ORC_INVALID_ARG;
    if (dims[0] == 0 || dims[1] == 0 || (ndim == 3 && dims[2] == 0)) return ORC_INVALID_ARG;
    uint64_t nz = ndim == 3 ? dims[2] : 1;
    uint64_t n = dims[0] * dims[1] * nz;
    if (n >= (1ull << 31)) return ORC_INVALID_ARG;
    if (!(eb > 0.0) || !isfinite(eb) || (rel != 0 && rel != 1)) return ORC_INVALID_ARG;
    if (rbf_k != 0 && rbf_k != 3 && rbf_k != 5 && rbf_k != 7) return ORC_INVALID_ARG;
    if (rs_sweeps == 0) rs_sweeps = 1;
    int topo = !(flags & FLAG_NO_TOPO);
    if (cap < orc_compress_bound(ndim, dims)) return ORC_BUFFER_TOO_SMALL;

    orc_qparams qp;
    int st = orc_qparams_compute(a, n, rel, eb, &qp);
    if (st) return st;

    /* CD + RP before any lossy step (Section IV-A) */
    uint8_t* labels = NULL;
    int32_t* delta = NULL;
    uint64_t k = 0, kmin = 0, kmax = 0, ksad = 0;
    if (topo) {
        uint64_t d3[3] = {dims[0], dims[1], nz};
        labels = (uint8_t*)malloc(n);
        orc_critical_points(a, ndim, d3, labels);
        for (uint64_t i = 0; i < n; i++) {
            kmin += labels[i] == ORC_MIN;
            kmax += labels[i] == ORC_MAX;
            ksad += labels[i] == ORC_SAD;
        }
        delta = (int32_t*)malloc((kmin + kmax + 1) * sizeof(int32_t));
        k = orc_ranks(a, labels, n, &qp, delta);
    }

    /* QZ, then B + LZ + BE */
    int32_t* q = (int32_t*)malloc(n * sizeof(int32_t));
    for (uint64_t i = 0; i < n; i++) q[i] = orc_quantize(a[i], &qp);
    const int tiles = (flags & FLAG_TILE_BLOCKS) != 0;
    codec_t cd;
    if (tiles) {
        const uint64_t d3[3] = {dims[0], dims[1], nz};
        codec_encode_tiles(q, ndim, d3, &cd);
    } else {
        codec_encode(q, n, &cd);
    }
    const uint64_t sum_abs = linear_sum_abs(q, n);

    int32_t kk;
    float sigma, g[9];
    rbf_params(sum_abs, n, cdiv(n, L), orc_quantize(qp.vmin, &qp), orc_quantize(qp.vmax, &qp),
               rbf_k, rbf_sigma, &kk, &sigma, g);

    layout_t lo;
    field_layout(n, cd.nblk, topo, cd.pay_words, &lo);
    codec_t rc;
    memset(&rc, 0, sizeof(rc));
    uint64_t sub[5] = {0, 0, 0, 0, 0};
    uint64_t end = lo.end;
    if (topo) {
        codec_encode(delta, k, &rc);
        rank_layout(lo.s7, k, rc.pay_words, sub);
        end = sub[4];
    }

    memset(out, 0, end);
    uint8_t* h = out;
    put32(h + 0, MAGIC);
    put32(h + 4, tiles ? VERSION_TILES : VERSION);
    put32(h + 8, (uint32_t)ndim);
    put32(h + 12, L);
    put64(h + 16, dims[0]);
    put64(h + 24, dims[1]);
    put64(h + 32, nz);
    put32(h + 40, flags & (FLAG_NO_TOPO | FLAG_RBF_SOLVE));
    put32(h + 44, (uint32_t)rel);
    putf64(h + 48, eb);
    putf64(h + 56, qp.eps);
    put32(h + 64, f2u(qp.w_f));
    put32(h + 68, f2u(qp.r_f));
    put32(h + 72, f2u(qp.h_f));
    put32(h + 76, (uint32_t)qp.const_field);
    put32(h + 80, f2u(qp.vmin));
    put32(h + 84, f2u(qp.vmax));
    put32(h + 88, (uint32_t)kk);
    put32(h + 92, f2u(sigma));
    put32(h + 96, rs_sweeps);
    put64(h + 104, n);
    put64(h + 112, cd.nblk);
    put64(h + 120, kmin);
    put64(h + 128, kmax);
    put64(h + 136, ksad);
    put64(h + 144, sum_abs);
    put64(h + 152, lo.s1);
    put64(h + 160, lo.s2);
    put64(h + 168, lo.s4);
    put64(h + 176, lo.s6);
    put64(h + 184, lo.s5);
    put64(h + 192, topo ? lo.s7 : end);
    put64(h + 200, end);
    put64(h + 208, cd.pay_words);
    put32(h + 216, (uint32_t)rc.pay_words);
    for (int i = 0; i < 9; i++) put32(h + 220 + 4 * i, f2u(g[i]));

    memcpy(out + lo.s1, cd.cbits, 4 * cdiv(cd.nblk, 32));
    memcpy(out + lo.s2, cd.width, cd.nblk);
    memcpy(out + lo.s4, cd.first, 4 * cd.nblk);
    if (topo) {
        for (uint64_t i = 0; i < n; i++) {
            uint32_t wv = get32(out + lo.s6 + 4 * (i / 16));
            wv |= (uint32_t)labels[i] << (2 * (i % 16));
            put32(out + lo.s6 + 4 * (i / 16), wv);
        }
    }
    memcpy(out + lo.s5, cd.pay, 4 * cd.pay_words);
    if (topo) {
        memcpy(out + sub[0], rc.cbits, 4 * cdiv(rc.nblk, 32));
        memcpy(out + sub[1], rc.width, rc.nblk);
        memcpy(out + sub[2], rc.first, 4 * rc.nblk);
        memcpy(out + sub[3], rc.pay, 4 * rc.pay_words);
        codec_free(&rc);
    }
    *out_size = end;
    codec_free(&cd);
    free(q);
    free(labels);
    free(delta);
    return ORC_OK;
}

/* -------------------------------------------------------------- decompress */

/* Move x by k representable binary32 values (k > 0 up, k < 0 down) on the
 * ordered-integer line; this is "delta * eta" with eta the machine epsilon of
 * x's own binade, i.e. delta units in the last place (R12).  Returns 0 if the
 * result would not be finite. */
static int step_ulps(float x, int64_t k, float* res) {
    uint32_t b = f2u(x);
    int64_t o = (b & 0x80000000u) ? -(int64_t)(b & 0x7FFFFFFFu) : (int64_t)b;
    o += k;
    if (o >= 0x7F800000ll || o <= -0x7F800000ll) return 0;
    uint32_t nb = o >= 0 ? (uint32_t)o : (0x80000000u | (uint32_t)(-o));
    *res = u2f(nb);
    return 1;
}

typedef struct { uint64_t idx; float v; } upd_t;

/* Colour classes of the saddle rounds: (x + 2y) mod 5 in 2D, (x + 2y + 3z) mod 7
 * in 3D; returns the number of classes in *ncol. */
int orc_colour(int ndim, uint64_t x, uint64_t y, uint64_t z, int* ncol) {
    *ncol = ndim == 2 ? 5 : 7;
    return (int)((x + 2 * y + (ndim == 3 ? 3 * z : 0)) % (uint64_t)*ncol);
}

int orc_decompress(const uint8_t* in, uint64_t size, float* out, uint64_t n_out,
                   float* d0, float* d1, uint64_t stats[4]) {
    if (size < HDR) return ORC_CORRUPT;
    const uint32_t version = get32(in + 4);
    if (get32(in) != MAGIC || (version != VERSION && version != VERSION_TILES) || get32(in + 12) != L)
        return ORC_CORRUPT;
    const int tiles = version == VERSION_TILES;
    int ndim = (int)get32(in + 8);
    uint64_t dims[3] = {get64(in + 16), get64(in + 24), get64(in + 32)};
    uint32_t flags = get32(in + 40);
    int topo = !(flags & FLAG_NO_TOPO);
    orc_qparams qp;
    memset(&qp, 0, sizeof(qp));
    qp.eps = getf64(in + 56);
    qp.w_f = u2f(get32(in + 64));
    qp.r_f = u2f(get32(in + 68));
    qp.h_f = u2f(get32(in + 72));
    int32_t kk = (int32_t)get32(in + 88);
    const float sigma = u2f(get32(in + 92));
    const int solve = (flags & FLAG_RBF_SOLVE) != 0;
    uint32_t sweeps = get32(in + 96);
    uint64_t n = get64(in + 104), nblk = get64(in + 112);
    uint64_t kmin = get64(in + 120), kmax = get64(in + 128);
    uint64_t pay_words = get64(in + 208), rpay = get32(in + 216);
    float g[9];
    for (int i = 0; i < 9; i++) g[i] = u2f(get32(in + 220 + 4 * i));
    if ((ndim != 2 && ndim != 3) || dims[0] == 0 || dims[1] == 0 || dims[2] == 0) return ORC_CORRUPT;
    if (ndim == 2 && dims[2] != 1) return ORC_CORRUPT;
    if (n != dims[0] * dims[1] * dims[2] || n != n_out) return ORC_CORRUPT;
    if (nblk != (tiles ? orc_tile_blocks(ndim, dims) : cdiv(n, L))) return ORC_CORRUPT;
    if (kk != 3 && kk != 5 && kk != 7) return ORC_CORRUPT;
    /* a header this writer cannot produce marks a damaged stream (R7): every
     * field within the range compression gives it, every section offset equal
     * to the layout recomputed from the counts */
    if (flags > 3u || sweeps < 1u || sweeps > 16u) return ORC_CORRUPT;
    if (solve && !(isfinite(sigma) && sigma > 0.0f)) return ORC_CORRUPT;
    if (!(isfinite(qp.w_f) && qp.w_f > 0.0f) || !(isfinite(qp.h_f) && qp.h_f >= 0.0f)) return ORC_CORRUPT;
    if (dims[0] > n_out || dims[1] > n_out || dims[2] > n_out) return ORC_CORRUPT;
    if (kmin > cdiv(n, 2) || kmax > cdiv(n, 2) || (!topo && (kmin || kmax))) return ORC_CORRUPT;
    if (pay_words > nblk * (L + 1) || rpay > cdiv(kmin + kmax, L) * (L + 1)) return ORC_CORRUPT;
    layout_t lo;
    field_layout(n, nblk, topo, pay_words, &lo);
    if (get64(in + 152) != lo.s1 || get64(in + 160) != lo.s2 || get64(in + 168) != lo.s4 ||
        get64(in + 176) != lo.s6 || get64(in + 184) != lo.s5 || get64(in + 192) != (topo ? lo.s7 : lo.end))
        return ORC_CORRUPT;
    uint64_t sub[5];
    uint64_t k = kmin + kmax;
    uint64_t end = lo.end;
    if (topo) {
        rank_layout(lo.s7, k, rpay, sub);
        end = sub[4];
    }
    if (get64(in + 200) != end || end > size) return ORC_CORRUPT;

    /* BE^, LZ^ + B^ */
    int32_t* q = (int32_t*)malloc(n * sizeof(int32_t));
    const int bad = tiles ? codec_decode_tiles(in + lo.s2, (const int32_t*)(in + lo.s4),
                                               (const uint32_t*)(in + lo.s5), pay_words, ndim, dims, q)
                          : codec_decode(in + lo.s2, (const int32_t*)(in + lo.s4), (const uint32_t*)(in + lo.s5),
                                         pay_words, n, q);
    if (bad) { free(q); return ORC_CORRUPT; }
    /* QZ^ */
    float* F = out;
    for (uint64_t i = 0; i < n; i++) F[i] = orc_dequantize(q[i], &qp);
    free(q);
    if (d0) memcpy(d0, F, n * sizeof(float));
    if (stats) memset(stats, 0, 4 * sizeof(uint64_t));
    if (!topo) {
        if (d1) memcpy(d1, F, n * sizeof(float));
        return ORC_OK;
    }

    /* MD^: 2-bit map and the losslessly coded rank sequence */
    uint8_t* lab = (uint8_t*)malloc(n);
    uint64_t cmin = 0, cmax = 0;
    for (uint64_t i = 0; i < n; i++) {
        lab[i] = (uint8_t)((get32(in + lo.s6 + 4 * (i / 16)) >> (2 * (i % 16))) & 3u);
        cmin += lab[i] == ORC_MIN;
        cmax += lab[i] == ORC_MAX;
    }
    int32_t* delta = (int32_t*)malloc((k + 1) * sizeof(int32_t));
    if (cmin != kmin || cmax != kmax ||
        codec_decode(in + sub[1], (const int32_t*)(in + sub[2]), (const uint32_t*)(in + sub[3]),
                     rpay, k, delta)) {
        free(lab); free(delta); return ORC_CORRUPT;
    }

    uint64_t d3[3] = {dims[0], dims[1], dims[2]};
    uint64_t stride[3] = {1, dims[0], dims[0] * dims[1]};
    float* D0 = (float*)malloc(n * sizeof(float));
    memcpy(D0, F, n * sizeof(float));

    /* CP^ + RP^: extrema stencils on lost extrema, every read from D0 (Jacobi) */
    uint64_t pos = 0;
    for (uint64_t i = 0; i < n; i++) {
        int t = lab[i];
        if (t != ORC_MIN && t != ORC_MAX) continue;
        int32_t dl = delta[pos++];
        if (orc_classify(D0, ndim, d3, i) == t) continue;     /* preserved */
        uint64_t c[3] = {i % dims[0], (i / dims[0]) % dims[1], i / (dims[0] * dims[1])};
        float ext = 0.0f;
        int have = 0;
        for (int ax = 0; ax < ndim; ax++) {
            if (c[ax] > 0) {
                float u = D0[i - stride[ax]];
                if (!have || (t == ORC_MAX ? u > ext : u < ext)) ext = u;
                have = 1;
            }
            if (c[ax] + 1 < dims[ax]) {
                float u = D0[i + stride[ax]];
                if (!have || (t == ORC_MAX ? u > ext : u < ext)) ext = u;
                have = 1;
            }
        }
        float v;
        int ok = have && step_ulps(ext, t == ORC_MAX ? (int64_t)dl : -(int64_t)dl, &v);
        if (ok && fabsf(v - D0[i]) <= qp.h_f) {
            F[i] = v;
            if (stats) stats[0]++;
        } else if (stats) {
            stats[1]++;
        }
    }
    if (d1) memcpy(d1, F, n * sizeof(float));

    /* RS^: RBF refinement of lost saddles in deterministic colour rounds.  The
     * colour (x + 2y) mod 5 in 2D, (x + 2y + 3z) mod 7 in 3D, keeps same-colour
     * points at Manhattan distance >= 3, so within a colour no two candidates
     * share a neighbour; all reads use the field at the start of the colour and
     * accepted values are written afterwards (R18). */
    int r = kk / 2;
    int ncol;
    orc_colour(ndim, 0, 0, 0, &ncol);
    int rz = ndim == 3 ? r : 0;
    upd_t* upd = (upd_t*)malloc((n + 1) * sizeof(upd_t));
    /* with the literal interpolation: its weights at p, rounded to binary32 */
    float af[343];
    if (solve) {
        double ad[343];
        const int m = orc_rbf_solve(ndim, r, sigma, 0, 0, 0, ad);
        for (int e = 0; e < m; e++) af[e] = (float)ad[e];
    }
    for (uint32_t sw = 0; sw < sweeps; sw++) {
        for (int col = 0; col < ncol; col++) {
            uint64_t nupd = 0;
            for (uint64_t i = 0; i < n; i++) {
                if (lab[i] != ORC_SAD) continue;
                uint64_t c[3] = {i % dims[0], (i / dims[0]) % dims[1], i / (dims[0] * dims[1])};
                int nc;
                if (orc_colour(ndim, c[0], c[1], c[2], &nc) != col) continue;
                /* a saddle label is valid at interior points only (R8/R9); a
                 * damaged stream may carry one elsewhere: never refined */
                int inside = 1;
                for (int ax = 0; ax < ndim; ax++)
                    if (c[ax] == 0 || c[ax] + 1 >= d3[ax]) inside = 0;
                if (!inside) continue;
                if (orc_classify(F, ndim, d3, i) == ORC_SAD) continue;   /* not lost */
                float Fp = F[i];
                /* tolerance eps_RBF = min(0.1 h, half the smallest nonzero local gap) (R15) */
                float gmin = INFINITY;
                for (int ax = 0; ax < ndim; ax++) {
                    float u1 = F[i - stride[ax]], u2 = F[i + stride[ax]];
                    float g1 = fabsf(u1 - Fp), g2 = fabsf(u2 - Fp);
                    if (g1 > 0.0f && g1 < gmin) gmin = g1;
                    if (g2 > 0.0f && g2 < gmin) gmin = g2;
                }
                if (gmin == INFINITY) continue;
                /* normalised Gaussian kernel over N_r(p) \ {p}, fixed offset order (R14);
                 * with the literal interpolation and the ball inside the grid,
                 * the interpolant's value at p instead: sum alpha_e F(p + o_e) */
                int ball_in = 1;
                for (int ax = 0; ax < ndim; ax++)
                    if (c[ax] < (uint64_t)r || c[ax] + (uint64_t)r >= d3[ax]) ball_in = 0;
                float num = 0.0f, den = 0.0f;
                int e = 0;
                for (int dz = -rz; dz <= rz; dz++)
                    for (int dy = -r; dy <= r; dy++)
                        for (int dx = -r; dx <= r; dx++) {
                            int d2 = dx * dx + dy * dy + dz * dz;
                            if (d2 == 0 || d2 > r * r) continue;
                            int64_t x = (int64_t)c[0] + dx, y = (int64_t)c[1] + dy, z = (int64_t)c[2] + dz;
                            const int slot = e++;
                            if (x < 0 || y < 0 || z < 0 || x >= (int64_t)dims[0] ||
                                y >= (int64_t)dims[1] || z >= (int64_t)dims[2]) continue;
                            float gw = (solve && ball_in) ? af[slot] : g[d2 - 1];
                            float fv = F[(uint64_t)x + dims[0] * ((uint64_t)y + dims[1] * (uint64_t)z)];
                            float prod = gw * fv;
                            num = num + prod;
                            den = den + gw;
                        }
                float u = (solve && ball_in) ? num : num / den;
                float v;
                if (solve) {
                    v = u;   /* the unclamped variant: acceptance alone bounds the step */
                } else {
                    float capv = fminf(0.1f * qp.h_f, 0.5f * gmin);
                    float stp = u - Fp;
                    if (stp > capv) stp = capv;
                    if (stp < -capv) stp = -capv;
                    v = Fp + stp;
                }
                if (v == Fp) continue;
                /* acceptance: p becomes a saddle; no neighbour changes type except to
                 * its own original label (no new FP/FT, Section IV-B end); bound kept */
                F[i] = v;
                int ok = orc_classify(F, ndim, d3, i) == ORC_SAD;
                for (int ax = 0; ax < ndim && ok; ax++) {
                    for (int sgn = -1; sgn <= 1 && ok; sgn += 2) {
                        uint64_t nb = sgn < 0 ? i - stride[ax] : i + stride[ax];
                        int tn = orc_classify(F, ndim, d3, nb);
                        F[i] = Fp;
                        int to = orc_classify(F, ndim, d3, nb);
                        F[i] = v;
                        if (tn != to && tn != lab[nb]) ok = 0;
                    }
                }
                F[i] = Fp;
                if (ok && fabsf(v - D0[i]) <= qp.h_f) {
                    upd[nupd].idx = i;
                    upd[nupd].v = v;
                    nupd++;
                }
            }
            for (uint64_t j = 0; j < nupd; j++) F[upd[j].idx] = upd[j].v;
            if (stats) stats[2] += nupd;
        }
    }
    free(upd);
    free(D0);
    free(lab);
    free(delta);
    return ORC_OK;
}

/* ------------------------------------------------ FN / FP / FT (Section III-B) */

void orc_topo_errors(const uint8_t* a, const uint8_t* b, uint64_t n, uint64_t out[12]) {
    memset(out, 0, 12 * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) {
        int x = a[i], y = b[i];
        if (x == y) continue;
        if (x != ORC_R && y == ORC_R) out[0 * 4 + x]++;        /* FN */
        else if (x == ORC_R && y != ORC_R) out[1 * 4 + y]++;   /* FP */
        else out[2 * 4 + x]++;                                 /* FT */
    }
}
