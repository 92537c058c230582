// tsz_internal.h -- declarations shared by the kernel files and the C-ABI layer.
#pragma once

#include "tsz_common.cuh"

namespace tsz {

constexpr int RANK_TILE = 2048;   // entries per dense-rank tile

// ---- launch geometry (set by toposzp_set_tuning; never changes results)
struct Tuning {
    int cd_threads = 256;
    int cd_blocks_per_sm = 8;
    int rounds_blocks_per_sm = 0;   // CTAs per SM of the saddle rounds (1024 threads per SM): 0 = 1
    int dec_slack_tiles = 0;        // 0: a quarter of the fused decoder's resident CTAs
    int saddle_records = 0;         // >= 0: neighbourhood records in the saddle rounds; < 0: field reads
    int dec_split = 0;              // > 0: the decoder stages as separate launches instead of fused
    int rank_bitmap = 0;            // 0: key bitmaps (+ bin table) when they fit; 1: no bin table; < 0: the sort
    int cd_columns = 0;             // 0: z-column pass when the planes and its warp count allow; 1: when the planes allow; < 0: never
    int launch_overlap = 0;         // 0: programmatic dependent launches; < 0: plain stream ordering
};
extern Tuning g_tuning;

// Launch with programmatic stream serialisation (griddep_enter() in
// tsz_common.cuh).  A stream being captured into a graph, and every launch
// while the launch_overlap tuning is negative, get plain launches (full
// stream ordering).  The attribute relaxes only the ordering after a
// preceding kernel: after a memset or an event wait the launch waits for it
// as usual.  Errors also surface through cudaGetLastError, like those of a
// <<<>>> launch.
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool plain = g_tuning.launch_overlap < 0 || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
                       cs != cudaStreamCaptureStatusNone;
    cfg.attrs = at;
    cfg.numAttrs = plain ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// ---- workspace carving (all offsets 256-byte aligned)
struct CompressWs {
    uint64_t ctrl, desc, rdesc, os_small, os_desc_a, os_desc_b, listM, listm, tmpM, tmpm, agg, delta, end;
    uint32_t list_cap, ntiles, rank_tiles, agg_stride, os_tiles, os_stride;
    int G;
};
// pointers of the radix sort's workspace (histograms, digit bases, tile
// counters in the zeroed control region; two look-back descriptor buffers)
struct SortWs {
    uint32_t *hist, *base, *ctr, *desc_a, *desc_b;
    uint32_t stride, max_tiles;
};
struct DecompressWs {
    uint64_t ctrl, rdesc, flags, tile_w, tile_c, pay_pre, cp_pre, cp_idx, delta, newv, sad, sadv, end;
    uint32_t ntiles, rank_tiles, sad_cap;
};
CompressWs compress_ws(uint64_t n, uint64_t nb_fmt = 0);   // nb_fmt: blocks of format v2 (0: v1)
DecompressWs decompress_ws(uint64_t n);

// ---- compression launchers (tsz_compress.cu)
void launch_range_cd(const float* a, const Geo& g, Ctrl* c, uint32_t* labels, bool topo, int sms,
                     cudaStream_t st);
void launch_critical_points(const float* a, const Geo& g, uint32_t* labels, unsigned long long* counts,
                            int sms, cudaStream_t st);
void launch_qparams(Ctrl* c, int* status, cudaStream_t st);
void launch_encode_field(const float* a, const uint32_t* labels, Ctrl* c, uint2* tcnt, uint32_t* scratch,
                         uint64_t region_bytes, uint8_t* out, const Layout& lo, uint2* listM, uint2* listm, bool topo,
                         const Geo& g, uint32_t nb_fmt, bool tiles, int sms, int* status, cudaStream_t st);
void launch_ranks(Ctrl* c, uint2* listM, uint2* listm, uint2* tmpM, uint2* tmpm, uint64_t tmp_bytes,
                  const SortWs& sw, uint2* agg, uint32_t agg_stride, const uint2* tpre, int32_t* delta, int G,
                  int sms, int* status, cudaStream_t st);
void launch_encode_ranks(const int32_t* delta, Ctrl* c, uint2* tcnt, uint32_t* scratch, uint8_t* out,
                         uint64_t max_k, int sms, int* status, cudaStream_t st);
void launch_finalize(Ctrl* c, uint8_t* out, uint64_t* out_size, int32_t rbf_k, float rbf_sigma,
                     int* status, cudaStream_t st);

// ---- decompression launchers (tsz_decompress.cu)
void launch_parse_header(const uint8_t* in, uint64_t in_size, uint64_t n_out, Ctrl* c, int* status,
                         uint32_t test_hold, cudaStream_t st);
void launch_dec_offsets(const uint8_t* in, Ctrl* c, uint32_t* tile_w, uint32_t* tile_c,
                        unsigned long long* pay_pre, uint32_t* cp_pre, uint32_t* rtile_w, uint32_t ntiles, int sms,
                        int* status, cudaStream_t st);
void launch_decode_tiles(const uint8_t* in, Ctrl* c, float* out, const unsigned long long* pay_pre,
                         const uint32_t* cp_pre, uint32_t* cp_idx, uint64_t n, int sms, int* status,
                         cudaStream_t st);
void launch_decode_ranks(const uint8_t* in, Ctrl* c, const uint32_t* rpre, int32_t* delta, uint64_t max_k,
                         int sms, int* status, cudaStream_t st);
void launch_decode_fused(const uint8_t* in, Ctrl* c, float* out, const unsigned long long* pay_pre,
                         const uint32_t* cp_pre, const int32_t* delta, uint32_t* cp_idx, float* newv,
                         uint32_t* flags, uint32_t* sad, uint32_t sad_cap, uint32_t ntiles_dec, uint32_t h_bound,
                         int sms, int* status, cudaStream_t st);
cudaError_t launch_saddle_rounds(const uint8_t* in, Ctrl* c, float* out, const uint32_t* sad, uint32_t* sadb,
                                 float* sadv, uint32_t sad_cap, uint32_t* rec, uint64_t rec_bytes, int sms,
                                 int* status, cudaStream_t st);

// ---- analysis
void launch_topo_errors(const uint32_t* a, const uint32_t* b, uint64_t n, unsigned long long* out12,
                        int sms, cudaStream_t st);

}  // namespace tsz
