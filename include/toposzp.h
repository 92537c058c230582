/* toposzp.h -- C ABI of the GB300 TopoSZp compression library (sm_103a).
 *
 * TopoSZp (arXiv 2602.17552) is an error-bounded lossy compressor for 2D/3D
 * float32 scalar fields that keeps critical points (minima, maxima, saddles)
 * and their relative order.  Compression (Section IV-A) runs CD + RP (critical
 * point labels and per-bin ranks), then SZp's QZ (quantisation), B + LZ
 * (blocking + Lorenzo) and BE (fixed-length encoding); decompression
 * (Section IV-B) inverts SZp, then applies the extrema stencils (CP^ + RP^) and
 * the RBF saddle refinement (RS^) under the relaxed bound |a - a'| < 2 eps.
 *
 * Conventions for every call:
 *  - Pointers are DEVICE pointers unless the comment says "host".
 *  - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream).  The library allocates no memory and never
 *    synchronises: the caller owns every buffer (field, output, workspace,
 *    status word).
 *  - The returned status covers argument checks done on the host before any
 *    work is queued.  Errors found on the device (non-finite input, bound too
 *    small, corrupt stream, a bounded wait that ran out) are written to the
 *    caller's device word `*status` (0 = OK), to be read after the stream is
 *    synchronised; later kernels of the same call then skip their work.
 *  - Fields are row-major with dims[0] = nx the fastest axis; ndim is 2
 *    (dims[2] ignored, treated as 1) or 3.  A 1D signal is a 2D field with
 *    ny = 1.  The number of points n must be below 2^31.
 *  - `field`, `out` and `workspace` must be 16-byte aligned (any torch or
 *    cudaMalloc allocation is).
 */
#ifndef TOPOSZP_H
#define TOPOSZP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* toposzp_stream;   /* a cudaStream_t */

typedef enum {
    TOPOSZP_OK = 0,
    TOPOSZP_ERR_INVALID_ARG = 1,     /* bad pointer, size, ndim, eb, params */
    TOPOSZP_ERR_NONFINITE = 2,       /* NaN or Inf in the input field */
    TOPOSZP_ERR_EB_TOO_SMALL = 3,    /* eps < ~2^-20 max|a|: codes would not fit */
    TOPOSZP_ERR_BUFFER_TOO_SMALL = 4,/* output capacity or workspace too small */
    TOPOSZP_ERR_CORRUPT_STREAM = 5,  /* header / section / payload inconsistent */
    TOPOSZP_ERR_TIMEOUT = 6,         /* a bounded device wait gave up */
    TOPOSZP_ERR_CUDA = 7,            /* a CUDA launch or copy failed */
    TOPOSZP_ERR_UNSUPPORTED = 8      /* outside the library's limits (n >= 2^31) */
} toposzp_status;

typedef enum {
    TOPOSZP_EB_ABS = 0,   /* eps = eb (the paper's absolute bound, Section V-A) */
    TOPOSZP_EB_REL = 1    /* eps = eb * (max(a) - min(a)), value-range relative */
} toposzp_eb_mode;

/* flags */
#define TOPOSZP_NO_TOPO 1u   /* SZp only: no labels, ranks or fix-ups (Fig. 9 baseline) */
/* RS^ by the literal RBF interpolation of Section IV-B(3), Eqs.
 * RBF-interp-final and RBF-eval: the refined value at a lost saddle p whose
 * whole ball N_r(p) lies in the grid is sum_i alpha_i D^(q_i) over
 * q_i in N_r(p) \ {p}, alpha the weights at p of the Gaussian interpolant with
 * a constant term (they sum to one), solved in binary64 when the stream is
 * decoded; the step is not clamped (the acceptance checks alone bound it).
 * Points whose ball leaves the grid keep the normalised kernel, unclamped.
 * Without the flag: the normalised kernel with the step clamped to
 * min(0.1 h, half the smallest nonzero face gap).  Stored in the header; the
 * decoder follows the stream. */
#define TOPOSZP_RBF_SOLVE 2u
/* Format v2 (stream version 2): blocks are tiles of 32 points, 8 x 4 in 2D
 * and 4 x 4 x 2 in 3D (x fastest), in raster order over the block grid, in
 * place of 32 consecutive points (Section II-C's B + LZ, tile-shaped).  Per
 * block, of the residuals of q - q_0 along the block's element order and its
 * block-local 2D / 3D Lorenzo residuals, the set with the smaller widest
 * residual is coded (bit 7 of the block's width byte: 1 = Lorenzo); positions
 * outside the grid take the code of the nearest point inside.  Every other
 * section and every decoded value are those of format v1: the flag changes
 * only the coded size.  toposzp_inspect reports it in info->flags; the
 * decoder reads the version from the stream. */
#define TOPOSZP_TILE_BLOCKS 4u

typedef struct {
    uint32_t flags;       /* an OR of TOPOSZP_NO_TOPO, TOPOSZP_RBF_SOLVE, TOPOSZP_TILE_BLOCKS */
    uint32_t rs_sweeps;   /* passes over the saddle colour rounds; 0 means 1 */
    int32_t rbf_k;        /* RBF kernel size 3, 5 or 7; 0 = adaptive (Section IV-B(3)) */
    float rbf_sigma;      /* Gaussian width; 0 = adaptive in [0.5, 1] */
} toposzp_params;

/* Host.  flags 0, one sweep, adaptive RBF parameters. */
void toposzp_default_params(toposzp_params* p);

/* Host.  Human-readable name of a status code (static string). */
const char* toposzp_status_string(toposzp_status s);

/* Host.  Upper bound on the compressed size in bytes for these dims (0 if the
 * dims are invalid); out_capacity >= this guarantees no overflow. */
uint64_t toposzp_compress_bound(int ndim, const uint64_t dims[3]);

/* Host.  Device workspace bytes needed by toposzp_compress /
 * toposzp_decompress for a field of these dims (0 if invalid).  Worst case:
 * it covers fields where every other point is an extremum. */
uint64_t toposzp_compress_workspace_size(int ndim, const uint64_t dims[3]);
uint64_t toposzp_decompress_workspace_size(int ndim, const uint64_t dims[3]);
/* Host.  The larger of the two: one workspace that serves both calls. */
uint64_t toposzp_workspace_size(int ndim, const uint64_t dims[3]);

/* Compress one field (Section IV-A: CD + RP, QZ, B + LZ, BE).
 *   field        device float32[n], read only
 *   ndim, dims   host; grid shape, dims[0] fastest
 *   mode, eb     error bound (eb > 0, finite)
 *   params       host, may be NULL for the defaults
 *   out          device byte buffer of out_capacity >= toposzp_compress_bound
 *   out_size     device uint64, receives the stream length (0 on a device error)
 *   workspace    device scratch of ws_bytes >= toposzp_compress_workspace_size;
 *                its contents on entry do not matter and are clobbered
 *   status       device int32, set to 0 then to the first device error
 * Stream format v1 (little-endian): a 256-byte header -- magic "TSZP",
 * version, ndim, block length L = 32, dims, flags, bound mode and eb, eps, the
 * quantiser's w, 1/w and h, a constant-field flag, the value range, RBF k and
 * sigma, sweeps, n, block count, extremum and saddle counts, the sum of the
 * absolute residuals, section offsets, total size, payload word counts, RBF
 * weights -- then the sections, each 16-byte aligned: (1) the
 * constant-block bitmap, (2) block widths (1 byte each), (4) first codes
 * (int32 each), (6) critical-point labels (2 bits per point), (5) the blocks'
 * sign and magnitude planes, (7) the rank stream coded the same way.  (6) and
 * (7) are absent with TOPOSZP_NO_TOPO.  The paper's section order (Section
 * IV-A, Fig. 6), with the fixed-size sections first. */
toposzp_status toposzp_compress(const float* field, int ndim, const uint64_t dims[3],
                                toposzp_eb_mode mode, double eb, const toposzp_params* params,
                                void* out, uint64_t out_capacity, uint64_t* out_size,
                                void* workspace, uint64_t ws_bytes, int32_t* status,
                                toposzp_stream stream);

/* Host.  Parse the first 256 bytes of a stream (a host copy) and report its
 * shape and sizes.  Returns CORRUPT_STREAM if the header is not a valid
 * TopoSZp v1 header: a field outside the range compression writes, or a
 * section offset other than the layout its counts give (the same rules the
 * decompressor applies on the device); UNSUPPORTED if the field has 2^31
 * points or more. */
typedef struct {
    int ndim;
    uint64_t dims[3];
    uint64_t n;
    uint64_t total_size;       /* bytes of the whole stream */
    double eps;                /* absolute error bound used */
    uint32_t flags;
    uint64_t k_min, k_max, k_saddle;
    int32_t rbf_k;
    float rbf_sigma;
} toposzp_info;
toposzp_status toposzp_inspect(const void* header_host, uint64_t header_bytes, toposzp_info* info);

/* Decompress a stream (Section IV-B: BE^, LZ^ + B^, QZ^, MD^, CP^ + RP^, RS^).
 *   in, in_size  device stream bytes (in_size >= the stream's total size)
 *   out          device float32[n_out]; n_out must equal the stream's n
 *   workspace    device scratch of ws_bytes >= toposzp_decompress_workspace_size
 *   status       device int32 (0 = OK; CORRUPT_STREAM if the stream is bad)
 * The output satisfies |a - out| <= eps + h < 2 eps (Table I's eps_topo). */
toposzp_status toposzp_decompress(const void* in, uint64_t in_size, float* out, uint64_t n_out,
                                  void* workspace, uint64_t ws_bytes, int32_t* status,
                                  toposzp_stream stream);

/* Critical point detection alone (Section IV-A(1)) on any field.
 *   labels_packed  device uint32[ceil(n/16)] or NULL: point i's code at bits
 *                  2(i mod 16) of word i/16; r = 0, m = 1, s = 2, M = 3
 *   counts4        device uint64[4] or NULL: number of r, m, s, M points
 *   status         device int32 (NaN compares false: such points are regular) */
toposzp_status toposzp_critical_points(const float* field, int ndim, const uint64_t dims[3],
                                       uint32_t* labels_packed, uint64_t* counts4,
                                       int32_t* status, toposzp_stream stream);

/* Topological error counts between two packed label maps (Section III-B):
 * out12[kind*4 + type], kind 0 = false negative (a critical point of `orig`
 * that is regular in `dec`), 1 = false positive (indexed by the new type),
 * 2 = false type (indexed by the original type).  out12 is overwritten. */
toposzp_status toposzp_topo_errors(const uint32_t* labels_orig, const uint32_t* labels_dec,
                                   uint64_t n, uint64_t* out12, toposzp_stream stream);

/* Compress without any workspace from the caller.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory --
 * e.g. an in-situ hook inside a simulation whose device memory is entirely
 * owned by the simulation's own pool allocator, or a caller running while a
 * CUDA graph is being captured, where a cudaMalloc would break the capture.
 * Same arguments, results and stream semantics as toposzp_compress, minus the
 * workspace: the library uses a static device array of its own instead.
 *   - Fields of at most toposzp_noalloc_max_points() points (262,144: e.g.
 *     512 x 512, or a 1 MiB float32 field); larger ones return
 *     TOPOSZP_ERR_UNSUPPORTED before any work is queued.
 *   - The array (about 5.4 MB) is part of the library's image: every GPU that
 *     loads the library holds it until the process exits.
 *   - No cudaMalloc, cudaFree or other allocating call is made.  The first
 *     call on each device looks up the array's device address (with that
 *     device current); make that first call before any stream capture.
 *   - Every call, on any stream, shares the one array per device and clears
 *     the parts that must start at zero; calls whose GPU work overlaps in time
 *     race on it, so serialise them (one stream, or events). */
toposzp_status toposzp_compress_noalloc(const float* field, int ndim, const uint64_t dims[3],
                                        toposzp_eb_mode mode, double eb, const toposzp_params* params,
                                        void* out, uint64_t out_capacity, uint64_t* out_size,
                                        int32_t* status, toposzp_stream stream);

/* Host.  Largest field (points) toposzp_compress_noalloc accepts. */
uint64_t toposzp_noalloc_max_points(void);

/* Host.  Launch geometry chosen by the autotuner (no counterpart in the
 * paper; no effect on any output bit).  Process-wide, not thread-safe; zero
 * fields keep the defaults.  Returns INVALID_ARG for unsupported values.
 *   cd_threads           threads per CTA of the range + CD pass: 128, 256, 512
 *   cd_blocks_per_sm     its CTAs per SM: 1..32 (default 8)
 *   rounds_blocks_per_sm CTAs per SM of the cooperative saddle rounds, which
 *                        run 1024 threads per SM: 1, 2 or 4 (default 1)
 *   dec_slack_tiles      extra lag, in 8192-point tiles, between the stages of
 *                        the fused decoder: 1..65536 (default: a quarter of its
 *                        resident CTAs)
 *   saddle_records       0 or 1: the saddle rounds copy each candidate's
 *                        neighbourhood into a compact record first (default);
 *                        -1: they read the field directly
 *   dec_split            0: one fused wavefront kernel decodes (default);
 *                        1: its four stages run as separate launches
 *   rank_bitmap          0: dense ranks from bitmaps over the key span when
 *                        they fit the workspace, else a radix sort, with a
 *                        table of each QZ bin's first rank when the bins of
 *                        the field's range fit (default); 1: the bitmaps
 *                        without that table; -1: always the radix sort
 *   cd_columns           0: the range + CD pass of 3D fields walks z-columns
 *                        when each plane is a whole number of 128-point
 *                        chunks and the columns, cut into segments of 4 to
 *                        32 planes, give at least 24 warps per SM (default);
 *                        1: whenever the planes allow; -1: never
 *   launch_overlap       0: each kernel is launched as a programmatic
 *                        dependent of the one before it on the stream, so
 *                        that its CTAs are scheduled while that one ends and
 *                        wait on the device for its results (default; plain
 *                        launches inside a stream capture); -1: plain
 *                        stream-ordered launches */
typedef struct {
    int32_t cd_threads;
    int32_t cd_blocks_per_sm;
    int32_t rounds_blocks_per_sm;
    int32_t dec_slack_tiles;
    int32_t saddle_records;
    int32_t dec_split;
    int32_t rank_bitmap;
    int32_t cd_columns;
    int32_t launch_overlap;
} toposzp_tuning;
toposzp_status toposzp_set_tuning(const toposzp_tuning* t);

/* Host.  Launch geometry for one size class of fields (no counterpart in the
 * paper; no effect on any output bit).  Size classes by the number of points
 * n: 0 for n < 2^16, 1 below 2^20, 2 below 2^24, 3 from 2^24.  Every call
 * picks the setting of its (ndim, class) when one was given, else the one
 * of toposzp_set_tuning; a decompression takes the 3D row of its class (the
 * stream's dimension is read on the device only).  t = NULL clears the
 * class.  Same value rules as toposzp_set_tuning; process-wide, not
 * thread-safe. */
toposzp_status toposzp_set_tuning_class(int ndim, int size_class, const toposzp_tuning* t);

/* Host.  The size class of a field of these dims (-1 if the dims are invalid). */
int toposzp_tuning_class(int ndim, const uint64_t dims[3]);

/* Host.  The launch geometry a compression of these dims would use. */
toposzp_status toposzp_get_tuning(int ndim, const uint64_t dims[3], toposzp_tuning* t);

/* ---- Batched form (no counterpart in the paper).  Many uneven fields in one
 * CUDA-graph replay: a plan fixes the fields' shapes, bounds and parameters and
 * spreads them over parallel branch streams (longest first onto the
 * least-loaded branch); a call forks the branches from `stream`, runs every
 * field's ordinary compress / decompress launch sequence on its branch, and
 * joins them.  The first call with a given set of pointers is captured into a
 * CUDA graph, later calls with the same pointers replay it; inside a caller's
 * own stream capture the launches are issued directly.  Outputs are
 * bit-identical to per-field toposzp_compress / toposzp_decompress.
 *
 * toposzp_batch_plan_create (host): nfields >= 1; ndims[i] in {2, 3};
 *   dims3[3i..3i+2] the field's dims (x fastest); modes / ebs per field;
 *   params (host, NULL = defaults) shared by all fields; tune_json (host, may
 *   be NULL) a JSON object whose "branches" member sets the branch count
 *   (default 8, at most nfields).  *plan receives an opaque handle.
 * toposzp_batch_workspace_size (host): bytes of workspace a call needs.
 * toposzp_batch_compress: fields[i] (host array of device pointers) in,
 *   outs[i] device buffers of at least toposzp_compress_bound bytes,
 *   out_sizes device uint64[nfields], statuses device int32[nfields].
 * toposzp_batch_decompress: ins[i] device buffers holding the streams (at least
 *   toposzp_compress_bound bytes each, e.g. the outs of a batch compress),
 *   outs[i] device float32[n_i], statuses device int32[nfields].
 * A plan serialises its own calls (one at a time, any thread); it must not be
 * destroyed while a call of it may still run on the device. */
toposzp_status toposzp_batch_plan_create(int nfields, const int* ndims, const uint64_t* dims3,
                                         const toposzp_eb_mode* modes, const double* ebs,
                                         const toposzp_params* params, const char* tune_json, void** plan);
uint64_t toposzp_batch_workspace_size(const void* plan);
int toposzp_batch_branches(const void* plan);
toposzp_status toposzp_batch_compress(void* plan, const float* const* fields, void* const* outs, uint64_t* out_sizes,
                                      void* workspace, uint64_t ws_bytes, int32_t* statuses, toposzp_stream stream);
toposzp_status toposzp_batch_decompress(void* plan, const void* const* ins, float* const* outs, void* workspace,
                                        uint64_t ws_bytes, int32_t* statuses, toposzp_stream stream);
void toposzp_batch_plan_destroy(void* plan);

/* Host.  Profiling hook (no counterpart in the paper).  After a call with
 * count > 0, every toposzp_compress records events[0..4] (cudaEvent_t handles
 * owned by the caller) on its stream: before the range + CD kernel, after it,
 * after the field encoder, after the rank stages, at the end; and every
 * toposzp_decompress records events[5..8]: at the start, after the header,
 * offsets and rank-stream decode, after the fused field decoder, at the end
 * (after the saddle rounds).  count must be 0 (off) or 9.
 * The setting is process-wide and not thread-safe; it is meant for a
 * single-threaded benchmark. */
toposzp_status toposzp_set_stage_events(void* const* events, int count);

/* Failure-path test hook (Section IV-B decoder; no effect unless set).  With
 * tile >= 0, the fused decoder of later toposzp_decompress calls never
 * publishes that 8192-point tile's decode stage: the stage waits that depend
 * on it run out their bounded spin, the call finishes with
 * TOPOSZP_ERR_TIMEOUT in its status word, and the context stays usable.  No
 * access leaves its buffer on that path (every position read from the
 * workspace is checked against n).  tile = -1 (the default) turns it off.
 * The decoder's split form (tuning dec_split = 1) has no waits and ignores it.
 * For tests only: the setting is process-wide, so while it is set every
 * toposzp_decompress of the process (any thread or stream) times out, and
 * toposzp_batch_decompress refuses to run (INVALID_ARG) rather than capture
 * the hold into its graph.  Reads and writes of the setting are atomic. */
toposzp_status toposzp_set_test_hold(int32_t tile);

#ifdef __cplusplus
}
#endif
#endif /* TOPOSZP_H */
