// tsz_api.cu -- the extern "C" entry points declared in include/toposzp.h.
//
// Host side only: argument validation, carving of the caller's workspace, and
// the launch sequence.  No allocation, no synchronisation, no host reads of
// device data; every data-dependent size is consumed on the device.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/toposzp.h"
#include "tsz_internal.h"

namespace tsz {

Tuning g_tuning;

constexpr uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

constexpr uint64_t CTRL_BYTES = 4096;
constexpr int SORT_G = 256;    // CTAs per list in the rank sort (fixed: sizes the workspace)

static_assert(sizeof(Ctrl) <= CTRL_BYTES, "control block too large");

static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 148;
    return sms;
}

static bool make_geo(int ndim, const uint64_t dims[3], Geo& g) {
    if (!dims || (ndim != 2 && ndim != 3)) return false;
    uint64_t nx = dims[0], ny = dims[1], nz = ndim == 3 ? dims[2] : 1;
    if (nx == 0 || ny == 0 || nz == 0) return false;
    if (nx >= (1ull << 31) || ny >= (1ull << 31) || nz >= (1ull << 31)) return false;
    uint64_t nxy = nx * ny;
    if (nxy >= (1ull << 31) || nxy * nz >= (1ull << 31)) return false;
    g.ndim = ndim;
    g.nx = (uint32_t)nx;
    g.ny = (uint32_t)ny;
    g.nz = (uint32_t)nz;
    g.nxy = (uint32_t)nxy;
    g.n = (uint32_t)(nxy * nz);
    g.nb = (uint32_t)cdiv(g.n, L);
    geo_divs(g);
    return true;
}

// nb_fmt: the blocks of a format-v2 stream (0 for format v1): the encoder's
// tiles then cover the larger of its payload tiles and the linear tiles
constexpr CompressWs compress_ws_c(uint64_t n, uint64_t nb_fmt = 0) {
    CompressWs w{};
    const uint64_t nb = cdiv(n, L) > nb_fmt ? cdiv(n, L) : nb_fmt;
    w.G = SORT_G;
    w.list_cap = (uint32_t)(cdiv(n, 2) + 1);
    w.ntiles = (uint32_t)cdiv(nb, TILE_BLOCKS);
    w.rank_tiles = (uint32_t)cdiv(cdiv(n + 2, L), TILE_BLOCKS) + 1;
    w.agg_stride = (uint32_t)cdiv(w.list_cap, RANK_TILE) + 1;
    w.os_tiles = (uint32_t)cdiv(w.list_cap, 4096);
    w.os_stride = w.os_tiles * 512u;   // up to 512 digits per tile
    uint64_t o = 0;
    w.ctrl = o; o = a256(o + CTRL_BYTES);
    w.desc = o; o = a256(o + 16ull * (w.ntiles + 1));   // per-tile counts, then prefixes
    w.rdesc = o; o = a256(o + 16ull * (w.rank_tiles + 1));
    w.os_small = o; o = a256(o + 4ull * (2 * 4 * 512) * 2 + 4ull * 8);   // histograms, bases, counters
    // end of the region zeroed at the start of every call
    w.os_desc_a = o; o = a256(o + 4ull * 2 * w.os_stride);
    w.os_desc_b = o; o = a256(o + 4ull * 2 * w.os_stride);
    w.listM = o; o = a256(o + 8ull * w.list_cap);
    w.listm = o; o = a256(o + 8ull * w.list_cap);
    w.tmpM = o; o = a256(o + 8ull * w.list_cap);
    w.tmpm = o; o = a256(o + 8ull * w.list_cap);
    // the encoder's per-tile payload slots share the sort's buffers (used later)
    const uint64_t slots = 4ull * (ENC_TILE_BLOCKS * 33) * cdiv(nb, ENC_TILE_BLOCKS);
    if (w.tmpM + slots > o) o = a256(w.tmpM + slots);
    w.agg = o; o = a256(o + 8ull * 2 * w.agg_stride);
    w.delta = o; o = a256(o + 4ull * (n + 2));
    w.end = o;
    return w;
}

CompressWs compress_ws(uint64_t n, uint64_t nb_fmt) { return compress_ws_c(n, nb_fmt); }

DecompressWs decompress_ws(uint64_t n) {
    DecompressWs w;
    const uint64_t nb = cdiv(n, L);
    w.ntiles = (uint32_t)cdiv(nb, 256);   // the fused decoder's 8192-point tiles
    // Per-tile counts and prefixes cover the linear tiles and the payload
    // tiles (256 blocks) of either format: a format-v2 stream has at most n
    // blocks, whatever the grid's shape (the host does not know it here).
    const uint64_t tcap = hmax<uint64_t>(w.ntiles, cdiv(n, 256));
    w.rank_tiles = (uint32_t)cdiv(cdiv(n + 2, L), TILE_BLOCKS) + 1;
    w.sad_cap = (uint32_t)n;
    uint64_t o = 0;
    w.ctrl = o; o = a256(o + CTRL_BYTES);
    w.rdesc = o; o = a256(o + 16ull * (w.rank_tiles + 1));
    w.flags = o; o = a256(o + 4ull * (w.ntiles + 1));
    w.tile_w = o; o = a256(o + 4ull * (tcap + 1));
    w.tile_c = o; o = a256(o + 4ull * (tcap + 1));
    w.pay_pre = o; o = a256(o + 8ull * (tcap + 1));
    w.cp_pre = o; o = a256(o + 4ull * (tcap + 1));
    w.cp_idx = o; o = a256(o + 4ull * (n + 2));
    w.delta = o; o = a256(o + 4ull * (n + 2));
    w.newv = o; o = a256(o + 4ull * (n + 2));
    w.sad = o; o = a256(o + 4ull * (n + 1));
    w.sadv = o; o = a256(o + 4ull * (n + 1));
    w.end = o;
    return w;
}

__global__ void k_init_ctrl(Ctrl* c, Geo g, int rel, double eb, uint32_t flags, int sweeps, uint32_t nb_fmt) {
    griddep_enter();
    c->g = g;
    c->nb_fmt = nb_fmt;
    c->rel = rel;
    c->eb = eb;
    c->flags = flags;
    c->rs_sweeps = sweeps;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static cudaEvent_t g_stage_ev[9];
static bool g_stage_on = false;
// toposzp_set_test_hold: the decode tile never published (-1: none).  Atomic:
// any thread's decompress may read it while a test sets it.
static std::atomic<int32_t> g_test_hold{-1};
static void stage(int i, cudaStream_t st) {
    if (g_stage_on) cudaEventRecord(g_stage_ev[i], st);
}


// Launch geometry per (ndim, size class), picked at the start of every call:
// the class's setting when one was given, else the process-wide default.  A
// decompression takes the 3D row of its class (the field's dimension is
// known on the device only).
static Tuning g_default;
static Tuning g_class[2][4];
static bool g_class_set[2][4];

static int size_class(uint64_t n) { return n < (1ull << 16) ? 0 : n < (1ull << 20) ? 1 : n < (1ull << 24) ? 2 : 3; }

static void select_tuning(int ndim, uint64_t n) {
    const int d = ndim == 3 ? 1 : 0, k = size_class(n);
    g_tuning = g_class_set[d][k] ? g_class[d][k] : g_default;
}

static bool make_tuning(const toposzp_tuning* t, Tuning& u) {
    if (t->cd_threads && t->cd_threads != 128 && t->cd_threads != 256 && t->cd_threads != 512) return false;
    if (t->cd_blocks_per_sm < 0 || t->cd_blocks_per_sm > 32) return false;
    if (t->rounds_blocks_per_sm != 0 && t->rounds_blocks_per_sm != 1 && t->rounds_blocks_per_sm != 2 &&
        t->rounds_blocks_per_sm != 4)
        return false;
    if (t->dec_slack_tiles < 0 || t->dec_slack_tiles > 65536) return false;
    if (t->saddle_records < -1 || t->saddle_records > 1) return false;
    if (t->dec_split < 0 || t->dec_split > 1) return false;
    if (t->rank_bitmap < -1 || t->rank_bitmap > 1) return false;
    if (t->cd_columns < -1 || t->cd_columns > 1) return false;
    if (t->launch_overlap < -1 || t->launch_overlap > 0) return false;
    u = Tuning();
    if (t->cd_threads) u.cd_threads = t->cd_threads;
    if (t->cd_blocks_per_sm) u.cd_blocks_per_sm = t->cd_blocks_per_sm;
    u.rounds_blocks_per_sm = t->rounds_blocks_per_sm;
    u.dec_slack_tiles = t->dec_slack_tiles;
    u.saddle_records = t->saddle_records;
    u.dec_split = t->dec_split;
    u.rank_bitmap = t->rank_bitmap;
    u.cd_columns = t->cd_columns;
    u.launch_overlap = t->launch_overlap;
    return true;
}

static void export_tuning(const Tuning& u, toposzp_tuning* t) {
    t->cd_threads = u.cd_threads;
    t->cd_blocks_per_sm = u.cd_blocks_per_sm;
    t->rounds_blocks_per_sm = u.rounds_blocks_per_sm;
    t->dec_slack_tiles = u.dec_slack_tiles;
    t->saddle_records = u.saddle_records;
    t->dec_split = u.dec_split;
    t->rank_bitmap = u.rank_bitmap;
    t->cd_columns = u.cd_columns;
    t->launch_overlap = u.launch_overlap;
}


// ------------------------------------------------ allocation-free compress
//
// Scratch for toposzp_compress_noalloc: a file-scope device array sized for
// the largest field that entry point accepts.  Every GPU that loads this
// library holds it until the process exits.  Host code never uses the array's
// name as an address: the device address is looked up once per device.
constexpr uint64_t NOALLOC_MAX_POINTS = 1ull << 18;
constexpr uint64_t NOALLOC_WS_BYTES = compress_ws_c(NOALLOC_MAX_POINTS).end;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_WS_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (set-up on the
// first call per device, with that device current).
static toposzp_status noalloc_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOPOSZP_ERR_CUDA;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return TOPOSZP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TOPOSZP_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return TOPOSZP_OK;
}

bool test_hold_active() { return g_test_hold.load() >= 0; }

}  // namespace tsz

using namespace tsz;

extern "C" {

void toposzp_default_params(toposzp_params* p) {
    if (!p) return;
    p->flags = 0;
    p->rs_sweeps = 1;
    p->rbf_k = 0;
    p->rbf_sigma = 0.0f;
}

const char* toposzp_status_string(toposzp_status s) {
    switch (s) {
        case TOPOSZP_OK: return "ok";
        case TOPOSZP_ERR_INVALID_ARG: return "invalid argument";
        case TOPOSZP_ERR_NONFINITE: return "non-finite value in the input field";
        case TOPOSZP_ERR_EB_TOO_SMALL: return "error bound too small for the field's magnitude";
        case TOPOSZP_ERR_BUFFER_TOO_SMALL: return "output buffer or workspace too small";
        case TOPOSZP_ERR_CORRUPT_STREAM: return "corrupt or mismatched compressed stream";
        case TOPOSZP_ERR_TIMEOUT: return "a bounded device wait timed out";
        case TOPOSZP_ERR_CUDA: return "CUDA launch or copy failed";
        case TOPOSZP_ERR_UNSUPPORTED: return "outside the supported limits";
    }
    return "unknown status";
}

uint64_t toposzp_compress_bound(int ndim, const uint64_t dims[3]) {
    Geo g;
    if (!make_geo(ndim, dims, g)) return 0;
    const uint64_t n = g.n, nb = hmax<uint64_t>(g.nb, tile_blocks(ndim, g.nx, g.ny, g.nz)), nbd = cdiv(n + 2, L);
    return HDR + 16 * 10 + 4 * cdiv(nb, 32) + nb + 4 * nb + 4 * cdiv(n, 16) + 4 * (L + 1) * nb +
           4 * cdiv(nbd, 32) + nbd + 4 * nbd + 4 * (L + 1) * nbd;
}

uint64_t toposzp_compress_workspace_size(int ndim, const uint64_t dims[3]) {
    Geo g;
    if (!make_geo(ndim, dims, g)) return 0;
    return hmax<uint64_t>(compress_ws(g.n).end, compress_ws(g.n, tile_blocks(ndim, g.nx, g.ny, g.nz)).end);
}

uint64_t toposzp_decompress_workspace_size(int ndim, const uint64_t dims[3]) {
    Geo g;
    if (!make_geo(ndim, dims, g)) return 0;
    return decompress_ws(g.n).end;
}

uint64_t toposzp_workspace_size(int ndim, const uint64_t dims[3]) {
    const uint64_t a = toposzp_compress_workspace_size(ndim, dims), b = toposzp_decompress_workspace_size(ndim, dims);
    return a > b ? a : b;
}

toposzp_status toposzp_compress(const float* field, int ndim, const uint64_t dims[3],
                                toposzp_eb_mode mode, double eb, const toposzp_params* params,
                                void* out, uint64_t out_capacity, uint64_t* out_size, void* workspace,
                                uint64_t ws_bytes, int32_t* status, toposzp_stream stream) {
    Geo g;
    if (!dims || (ndim != 2 && ndim != 3)) return TOPOSZP_ERR_INVALID_ARG;
    if (!make_geo(ndim, dims, g)) {
        const uint64_t nz = ndim == 3 ? dims[2] : 1;
        if (dims[0] && dims[1] && nz) return TOPOSZP_ERR_UNSUPPORTED;
        return TOPOSZP_ERR_INVALID_ARG;
    }
    toposzp_params p;
    toposzp_default_params(&p);
    if (params) p = *params;
    if (p.rs_sweeps == 0) p.rs_sweeps = 1;
    if (!field || !out || !out_size || !workspace || !status) return TOPOSZP_ERR_INVALID_ARG;
    if (!aligned16(field) || !aligned16(out) || !aligned16(workspace)) return TOPOSZP_ERR_INVALID_ARG;
    if (mode != TOPOSZP_EB_ABS && mode != TOPOSZP_EB_REL) return TOPOSZP_ERR_INVALID_ARG;
    if (!(eb > 0.0) || !std::isfinite(eb)) return TOPOSZP_ERR_INVALID_ARG;
    if (p.flags & ~(TOPOSZP_NO_TOPO | TOPOSZP_RBF_SOLVE | TOPOSZP_TILE_BLOCKS)) return TOPOSZP_ERR_INVALID_ARG;
    if (p.rs_sweeps > 16) return TOPOSZP_ERR_INVALID_ARG;
    if (p.rbf_k != 0 && p.rbf_k != 3 && p.rbf_k != 5 && p.rbf_k != 7) return TOPOSZP_ERR_INVALID_ARG;
    if (!(p.rbf_sigma >= 0.0f) || !std::isfinite(p.rbf_sigma)) return TOPOSZP_ERR_INVALID_ARG;
    if (out_capacity < toposzp_compress_bound(ndim, dims)) return TOPOSZP_ERR_BUFFER_TOO_SMALL;
    const bool tiles = (p.flags & TOPOSZP_TILE_BLOCKS) != 0;
    const uint32_t nbf = tiles ? (uint32_t)tile_blocks(ndim, g.nx, g.ny, g.nz) : g.nb;
    const CompressWs w = compress_ws(g.n, tiles ? nbf : 0);
    if (ws_bytes < w.end) return TOPOSZP_ERR_BUFFER_TOO_SMALL;
    select_tuning(ndim, g.n);

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* ws = reinterpret_cast<uint8_t*>(workspace);
    uint8_t* o = reinterpret_cast<uint8_t*>(out);
    Ctrl* c = reinterpret_cast<Ctrl*>(ws + w.ctrl);
    uint2* tcnt = reinterpret_cast<uint2*>(ws + w.desc);
    uint2* listM = reinterpret_cast<uint2*>(ws + w.listM);
    uint2* listm = reinterpret_cast<uint2*>(ws + w.listm);
    const bool topo = !(p.flags & TOPOSZP_NO_TOPO);
    const int sms = sm_count();
    Layout lo;
    make_layout(g.n, nbf, topo, 0, 0, 0, lo);
    uint32_t* labels = reinterpret_cast<uint32_t*>(o + lo.s6);

    cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    cudaMemsetAsync(ws, 0, w.os_desc_a, st);   // control block, per-tile counts, sort histograms and counters
    launch_pdl(k_init_ctrl, dim3(1), dim3(1), 0, st, c, g, mode == TOPOSZP_EB_REL ? 1 : 0, eb, p.flags, (int)p.rs_sweeps, nbf);
    stage(0, st);
    launch_range_cd(field, g, c, labels, topo, sms, st);
    stage(1, st);
    launch_qparams(c, status, st);
    launch_encode_field(field, labels, c, tcnt, reinterpret_cast<uint32_t*>(ws + w.tmpM), w.agg - w.tmpM, o, lo,
                        listM, listm, topo, g, nbf, tiles, sms, status, st);
    stage(2, st);
    if (topo) {
        SortWs sw;
        sw.hist = reinterpret_cast<uint32_t*>(ws + w.os_small);
        sw.base = sw.hist + 2 * 4 * 512;
        sw.ctr = sw.base + 2 * 4 * 512;
        sw.desc_a = reinterpret_cast<uint32_t*>(ws + w.os_desc_a);
        sw.desc_b = reinterpret_cast<uint32_t*>(ws + w.os_desc_b);
        sw.stride = w.os_stride;
        sw.max_tiles = w.os_tiles;
        launch_ranks(c, listM, listm, reinterpret_cast<uint2*>(ws + w.tmpM),
                     reinterpret_cast<uint2*>(ws + w.tmpm), w.agg - w.tmpM, sw, reinterpret_cast<uint2*>(ws + w.agg),
                     w.agg_stride, tcnt, reinterpret_cast<int32_t*>(ws + w.delta), w.G, sms, status, st);
        // the rank payload slots reuse the sort's buffers (free again by now)
        launch_encode_ranks(reinterpret_cast<int32_t*>(ws + w.delta), c, reinterpret_cast<uint2*>(ws + w.rdesc),
                            reinterpret_cast<uint32_t*>(ws + w.tmpM), o, g.n, sms, status, st);
    }
    stage(3, st);
    launch_finalize(c, o, out_size, p.rbf_k, p.rbf_sigma, status, st);
    stage(4, st);
    return cudaGetLastError() == cudaSuccess ? TOPOSZP_OK : TOPOSZP_ERR_CUDA;
}

toposzp_status toposzp_compress_noalloc(const float* field, int ndim, const uint64_t dims[3],
                                        toposzp_eb_mode mode, double eb, const toposzp_params* params,
                                        void* out, uint64_t out_capacity, uint64_t* out_size,
                                        int32_t* status, toposzp_stream stream) {
    Geo g;
    if (!dims || (ndim != 2 && ndim != 3)) return TOPOSZP_ERR_INVALID_ARG;
    if (!make_geo(ndim, dims, g)) {   // the same split as toposzp_compress
        const uint64_t nz = ndim == 3 ? dims[2] : 1;
        return dims[0] && dims[1] && nz ? TOPOSZP_ERR_UNSUPPORTED : TOPOSZP_ERR_INVALID_ARG;
    }
    if (g.n > NOALLOC_MAX_POINTS) return TOPOSZP_ERR_UNSUPPORTED;   // larger than the static scratch
    void* scratch = nullptr;
    const toposzp_status st = noalloc_scratch(&scratch);
    if (st != TOPOSZP_OK) return st;
    return toposzp_compress(field, ndim, dims, mode, eb, params, out, out_capacity, out_size, scratch,
                            NOALLOC_WS_BYTES, status, stream);
}

uint64_t toposzp_noalloc_max_points(void) { return NOALLOC_MAX_POINTS; }

toposzp_status toposzp_inspect(const void* header_host, uint64_t header_bytes, toposzp_info* info) {
    if (!header_host || !info || header_bytes < HDR) return TOPOSZP_ERR_INVALID_ARG;
    const uint8_t* h = reinterpret_cast<const uint8_t*>(header_host);
    auto u32 = [&](int off) { uint32_t v; std::memcpy(&v, h + off, 4); return v; };
    auto u64 = [&](int off) { uint64_t v; std::memcpy(&v, h + off, 8); return v; };
    const uint32_t version = u32(4);
    if (u32(0) != MAGIC || (version != VERSION && version != VERSION_TILES) || u32(12) != L)
        return TOPOSZP_ERR_CORRUPT_STREAM;
    std::memset(info, 0, sizeof(*info));
    info->ndim = (int)u32(8);
    info->dims[0] = u64(16);
    info->dims[1] = u64(24);
    info->dims[2] = u64(32);
    if ((info->ndim != 2 && info->ndim != 3) || !info->dims[0] || !info->dims[1] || !info->dims[2])
        return TOPOSZP_ERR_CORRUPT_STREAM;
    if (info->ndim == 2 && info->dims[2] != 1) return TOPOSZP_ERR_CORRUPT_STREAM;
    for (int d = 0; d < 3; d++)
        if (info->dims[d] >= (1ull << 31)) return TOPOSZP_ERR_UNSUPPORTED;
    info->n = u64(104);
    if (info->n != info->dims[0] * info->dims[1] * info->dims[2]) return TOPOSZP_ERR_CORRUPT_STREAM;
    if (info->n >= (1ull << 31)) return TOPOSZP_ERR_UNSUPPORTED;
    // every other field within the range compression writes, and the section
    // offsets equal to the layout recomputed from the counts (the same rules
    // as the device-side header check)
    const uint64_t n = info->n, nb = u64(112), kmin = u64(120), kmax = u64(128);
    const uint64_t pay = u64(208), rpay = u32(216);
    const uint32_t flags = u32(40), sweeps = u32(96);
    const int32_t rk = (int32_t)u32(88);
    float w_f, h_f;
    std::memcpy(&w_f, h + 64, 4);
    std::memcpy(&h_f, h + 72, 4);
    const bool topo = !(flags & TOPOSZP_NO_TOPO);
    float sigma;
    std::memcpy(&sigma, h + 92, 4);
    const uint64_t nb_want = version == VERSION_TILES
                                 ? tile_blocks(info->ndim, info->dims[0], info->dims[1], info->dims[2])
                                 : cdiv(n, L);
    bool ok = nb == nb_want && flags <= (TOPOSZP_NO_TOPO | TOPOSZP_RBF_SOLVE) && sweeps >= 1u && sweeps <= 16u;
    ok = ok && (!(flags & TOPOSZP_RBF_SOLVE) || (std::isfinite(sigma) && sigma > 0.0f));
    ok = ok && (rk == 3 || rk == 5 || rk == 7) && std::isfinite(w_f) && w_f > 0.0f && std::isfinite(h_f) &&
         h_f >= 0.0f;
    ok = ok && kmin <= cdiv(n, 2) && kmax <= cdiv(n, 2) && (topo || (kmin == 0 && kmax == 0));
    ok = ok && pay <= nb * (L + 1) && rpay <= cdiv(kmin + kmax, L) * (L + 1);
    if (!ok) return TOPOSZP_ERR_CORRUPT_STREAM;
    Layout lo;
    make_layout(n, nb, topo, pay, kmin + kmax, rpay, lo);
    if (lo.end != u64(200) || lo.s1 != u64(152) || lo.s2 != u64(160) || lo.s4 != u64(168) ||
        lo.s6 != u64(176) || lo.s5 != u64(184) || (topo ? lo.s7 : lo.end) != u64(192))
        return TOPOSZP_ERR_CORRUPT_STREAM;
    info->total_size = u64(200);
    std::memcpy(&info->eps, h + 56, 8);
    info->flags = u32(40) | (version == VERSION_TILES ? TOPOSZP_TILE_BLOCKS : 0u);
    info->k_min = u64(120);
    info->k_max = u64(128);
    info->k_saddle = u64(136);
    info->rbf_k = (int32_t)u32(88);
    std::memcpy(&info->rbf_sigma, h + 92, 4);
    return TOPOSZP_OK;
}

toposzp_status toposzp_decompress(const void* in, uint64_t in_size, float* out, uint64_t n_out,
                                  void* workspace, uint64_t ws_bytes, int32_t* status,
                                  toposzp_stream stream) {
    if (!in || !out || !workspace || !status || n_out == 0) return TOPOSZP_ERR_INVALID_ARG;
    if (n_out >= (1ull << 31)) return TOPOSZP_ERR_UNSUPPORTED;
    if (!aligned16(in) || !aligned16(out) || !aligned16(workspace)) return TOPOSZP_ERR_INVALID_ARG;
    const DecompressWs w = decompress_ws(n_out);
    if (ws_bytes < w.end) return TOPOSZP_ERR_BUFFER_TOO_SMALL;
    select_tuning(3, n_out);   // the 3D row: the dimension is known on the device only
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* ws = reinterpret_cast<uint8_t*>(workspace);
    const uint8_t* src = reinterpret_cast<const uint8_t*>(in);
    Ctrl* c = reinterpret_cast<Ctrl*>(ws + w.ctrl);
    const int sms = sm_count();
    cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    cudaMemsetAsync(ws, 0, w.tile_w, st);   // control block, rank tile sums, stage flags
    stage(5, st);
    launch_parse_header(src, in_size, n_out, c, status, (uint32_t)(g_test_hold.load() + 1), st);
    // the rank stream's tile sums and prefixes live in the (no longer used) rank descriptor region
    uint32_t* rtile = reinterpret_cast<uint32_t*>(ws + w.rdesc);
    launch_dec_offsets(src, c, reinterpret_cast<uint32_t*>(ws + w.tile_w), reinterpret_cast<uint32_t*>(ws + w.tile_c),
                       reinterpret_cast<unsigned long long*>(ws + w.pay_pre), reinterpret_cast<uint32_t*>(ws + w.cp_pre),
                       rtile, w.ntiles, sms, status, st);
    launch_decode_ranks(src, c, rtile, reinterpret_cast<int32_t*>(ws + w.delta), n_out, sms, status, st);
    // format v2's S1 (returns at once on a format-v1 stream, whose S1 is in the fused decoder)
    launch_decode_tiles(src, c, out, reinterpret_cast<unsigned long long*>(ws + w.pay_pre),
                        reinterpret_cast<uint32_t*>(ws + w.cp_pre), reinterpret_cast<uint32_t*>(ws + w.cp_idx), n_out,
                        sms, status, st);
    stage(6, st);
    launch_decode_fused(src, c, out, reinterpret_cast<unsigned long long*>(ws + w.pay_pre),
                        reinterpret_cast<uint32_t*>(ws + w.cp_pre), reinterpret_cast<int32_t*>(ws + w.delta),
                        reinterpret_cast<uint32_t*>(ws + w.cp_idx), reinterpret_cast<float*>(ws + w.newv),
                        reinterpret_cast<uint32_t*>(ws + w.flags), reinterpret_cast<uint32_t*>(ws + w.sad),
                        w.sad_cap, w.ntiles, 64u, sms, status, st);
    stage(7, st);
    // the stencil values are consumed by now: their buffer holds the colour
    // buckets; the extremum positions and ranks (contiguous) hold the records
    cudaError_t e = launch_saddle_rounds(src, c, out, reinterpret_cast<uint32_t*>(ws + w.sad),
                                         reinterpret_cast<uint32_t*>(ws + w.newv),
                                         reinterpret_cast<float*>(ws + w.sadv), w.sad_cap,
                                         reinterpret_cast<uint32_t*>(ws + w.cp_idx), w.newv - w.cp_idx, sms,
                                         status, st);
    if (e != cudaSuccess) return TOPOSZP_ERR_CUDA;
    stage(8, st);
    return cudaGetLastError() == cudaSuccess ? TOPOSZP_OK : TOPOSZP_ERR_CUDA;
}


toposzp_status toposzp_set_tuning_class(int ndim, int size_class_index, const toposzp_tuning* t) {
    if ((ndim != 2 && ndim != 3) || size_class_index < 0 || size_class_index > 3) return TOPOSZP_ERR_INVALID_ARG;
    const int d = ndim == 3 ? 1 : 0;
    if (!t) {
        g_class_set[d][size_class_index] = false;
        return TOPOSZP_OK;
    }
    Tuning u;
    if (!make_tuning(t, u)) return TOPOSZP_ERR_INVALID_ARG;
    g_class[d][size_class_index] = u;
    g_class_set[d][size_class_index] = true;
    return TOPOSZP_OK;
}

int toposzp_tuning_class(int ndim, const uint64_t dims[3]) {
    Geo g;
    if (!make_geo(ndim, dims, g)) return -1;
    return size_class(g.n);
}

toposzp_status toposzp_get_tuning(int ndim, const uint64_t dims[3], toposzp_tuning* t) {
    Geo g;
    if (!t || !make_geo(ndim, dims, g)) return TOPOSZP_ERR_INVALID_ARG;
    const int d = ndim == 3 ? 1 : 0, k = size_class(g.n);
    export_tuning(g_class_set[d][k] ? g_class[d][k] : g_default, t);
    return TOPOSZP_OK;
}

toposzp_status toposzp_set_tuning(const toposzp_tuning* t) {
    if (!t) return TOPOSZP_ERR_INVALID_ARG;
    Tuning u;
    if (!make_tuning(t, u)) return TOPOSZP_ERR_INVALID_ARG;
    g_default = u;
    g_tuning = u;
    return TOPOSZP_OK;
}

toposzp_status toposzp_set_test_hold(int32_t tile) {
    if (tile < -1) return TOPOSZP_ERR_INVALID_ARG;
    g_test_hold.store(tile);
    return TOPOSZP_OK;
}

toposzp_status toposzp_set_stage_events(void* const* events, int count) {
    if (count == 0) {
        g_stage_on = false;
        return TOPOSZP_OK;
    }
    if (count != 9 || !events) return TOPOSZP_ERR_INVALID_ARG;
    for (int i = 0; i < 9; i++) {
        if (!events[i]) return TOPOSZP_ERR_INVALID_ARG;
        g_stage_ev[i] = reinterpret_cast<cudaEvent_t>(events[i]);
    }
    g_stage_on = true;
    return TOPOSZP_OK;
}

toposzp_status toposzp_critical_points(const float* field, int ndim, const uint64_t dims[3],
                                       uint32_t* labels_packed, uint64_t* counts4, int32_t* status,
                                       toposzp_stream stream) {
    Geo g;
    if (!field || !status || (!labels_packed && !counts4)) return TOPOSZP_ERR_INVALID_ARG;
    if (!make_geo(ndim, dims, g)) return TOPOSZP_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(field) & 3u) || (reinterpret_cast<uintptr_t>(labels_packed) & 3u) ||
        (reinterpret_cast<uintptr_t>(counts4) & 7u))
        return TOPOSZP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (counts4) cudaMemsetAsync(counts4, 0, 4 * sizeof(uint64_t), st);
    launch_critical_points(field, g, labels_packed, reinterpret_cast<unsigned long long*>(counts4),
                           sm_count(), st);
    return cudaGetLastError() == cudaSuccess ? TOPOSZP_OK : TOPOSZP_ERR_CUDA;
}

toposzp_status toposzp_topo_errors(const uint32_t* labels_orig, const uint32_t* labels_dec, uint64_t n,
                                   uint64_t* out12, toposzp_stream stream) {
    if (!labels_orig || !labels_dec || !out12 || n == 0) return TOPOSZP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(out12, 0, 12 * sizeof(uint64_t), st);
    launch_topo_errors(labels_orig, labels_dec, n, reinterpret_cast<unsigned long long*>(out12), sm_count(),
                       st);
    return cudaGetLastError() == cudaSuccess ? TOPOSZP_OK : TOPOSZP_ERR_CUDA;
}

}  // extern "C"
