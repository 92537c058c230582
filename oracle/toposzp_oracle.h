/* TopoSZp CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C implementation of the TopoSZp method
 * (arXiv 2602.17552) used to check the CUDA library bit for bit.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it.  It shares no code or header with the CUDA
 * library: every constant and layout rule below is restated here on purpose.
 *
 * Compression stages follow Section IV-A in the paper's order: CD (critical
 * point detection), RP (relative positions), QZ (quantisation, Section II-C),
 * B+LZ (blocking + Lorenzo), BE (fixed-length byte encoding).  Decompression
 * follows Section IV-B: BE^, LZ^+B^, QZ^, MD^ (metadata), CP^+RP^ (extrema
 * stencils), RS^ (RBF saddle refinement).
 *
 * Parity unpinned: two constants of the RS^ reading, which the paper does not
 * give -- the step limit 0.1 h of eps_RBF, and the neighbour-variation
 * thresholds that pick sigma and the kernel size (Section IV-B(3)).  The tests
 * pin their stated properties and direction only; the kernel value, the
 * neighbourhood, its cut at the boundary and the acceptance rules are pinned
 * by hand-worked fixtures.
 */
#ifndef TOPOSZP_ORACLE_H
#define TOPOSZP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (values mirror the library's on purpose) */
enum { ORC_OK = 0, ORC_INVALID_ARG = 1, ORC_NONFINITE = 2, ORC_EB_TOO_SMALL = 3,
       ORC_BUFFER_TOO_SMALL = 4, ORC_CORRUPT = 5 };

/* labels (Section IV-A(1)): r=0 m=1 s=2 M=3 */
enum { ORC_R = 0, ORC_MIN = 1, ORC_SAD = 2, ORC_MAX = 3 };

typedef struct {
    float vmin, vmax;       /* value range of the field */
    double eps;             /* absolute error bound */
    float w_f, r_f, h_f;    /* bin width, its reciprocal, acceptance half-width */
    int const_field;        /* 1 when vmax == vmin */
} orc_qparams;

/* --- individual stages, exposed for stage-by-stage tests --- */
int  orc_qparams_compute(const float* a, uint64_t n, int rel, double eb, orc_qparams* p);
int32_t orc_quantize(float a, const orc_qparams* p);           /* QZ */
float   orc_dequantize(int32_t q, const orc_qparams* p);       /* QZ^ */
int  orc_classify(const float* a, int ndim, const uint64_t dims[3], uint64_t i);   /* CD */
void orc_critical_points(const float* a, int ndim, const uint64_t dims[3], uint8_t* labels);
/* RP: dense per-bin ranks of every m/M point, listed in increasing index order */
uint64_t orc_ranks(const float* a, const uint8_t* labels, uint64_t n, const orc_qparams* p,
                   int32_t* delta_seq);
double orc_exp_neg(double t);                                    /* exp(-t), t >= 0 */
/* Weights of the Gaussian RBF interpolant over the offsets of N_r(p) \ {p}
 * (table order: z, then y, then x ascending), evaluated at offset (ex, ey, ez)
 * from p: alpha = Phi^-1 phi, in binary64.  Returns the number of offsets. */
int orc_rbf_solve(int ndim, int r, float sigma, int ex, int ey, int ez, double* alpha);
int orc_colour(int ndim, uint64_t x, uint64_t y, uint64_t z, int* ncol);   /* RS^ rounds */

/* --- whole pipeline --- */
uint64_t orc_compress_bound(int ndim, const uint64_t dims[3]);   /* either format */
/* Blocks of format v2 (8 x 4 tiles in 2D, 4 x 4 x 2 in 3D) covering the grid. */
uint64_t orc_tile_blocks(int ndim, const uint64_t dims[3]);
/* rel: 0 absolute eb, 1 eb * (max - min).  flags bit0: no topology (SZp only);
 * bit1: RS^ by the literal RBF interpolation, unclamped (see orc_decompress);
 * bit2: format v2, tile-shaped blocks with block-local 2D / 3D Lorenzo
 * residuals (header version 2; the decoded field equals format v1's).
 * rbf_k / rbf_sigma: 0 = adaptive.  Returns a status; *out_size on success. */
int orc_compress(const float* a, int ndim, const uint64_t dims[3], int rel, double eb,
                 uint32_t flags, uint32_t rs_sweeps, int32_t rbf_k, float rbf_sigma,
                 uint8_t* out, uint64_t cap, uint64_t* out_size);
/* d0 / d1 (optional, n floats): snapshots after QZ^ and after CP^+RP^. */
int orc_decompress(const uint8_t* in, uint64_t size, float* out, uint64_t n,
                   float* d0, float* d1, uint64_t stats[4]);
/* FN/FP/FT per type, indexed [kind*4 + type] (kind 0 FN, 1 FP, 2 FT) */
void orc_topo_errors(const uint8_t* lab_a, const uint8_t* lab_b, uint64_t n, uint64_t out[12]);

#ifdef __cplusplus
}
#endif
#endif
