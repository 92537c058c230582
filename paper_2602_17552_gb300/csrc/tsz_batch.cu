// Batched form of the C ABI: many uneven fields compressed or decompressed in
// one replay of a CUDA graph.
//
// A plan fixes the fields' shapes, bounds and parameters.  The fields are
// spread over `branches` streams, longest first onto the least-loaded branch,
// so that small fields which leave most SMs idle run side by side; each branch
// owns one slice of the caller's workspace, sized for its largest field.  A
// call forks the branches from the caller's stream, issues every field's
// ordinary launch sequence (toposzp_compress / toposzp_decompress) on its
// branch, and joins them back.  The first call with a given set of pointers is
// captured into a CUDA graph; later calls with the same pointers replay it.
// Under a caller's own stream capture the launches are issued directly, so
// they land in the caller's graph.  Every field goes through exactly the same
// kernels as a plain call: the outputs are identical.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/toposzp.h"

namespace tsz {
bool test_hold_active();   // tsz_api.cu: the failure-path test hook is set
}

namespace {

constexpr uint64_t ALIGN = 256;
uint64_t up(uint64_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Field {
    int ndim;
    uint64_t dims[3];
    toposzp_eb_mode mode;
    double eb;
    uint64_t n, ws_c, ws_d, bound;
    int branch;
};

struct Plan {
    std::vector<Field> f;
    toposzp_params params;
    int branches = 1;
    std::vector<uint64_t> ws_off;   // per branch, into the caller's workspace
    uint64_t ws_bytes = 0;
    std::vector<cudaStream_t> st;
    cudaStream_t cap = nullptr;     // capture origin
    std::vector<cudaEvent_t> ev;    // [0] fork, [1..branches] joins
    // the captured graphs and the pointers they were captured with
    struct Cached {
        cudaGraphExec_t exec = nullptr;
        std::vector<const void*> key;
    } cached[2];
    std::mutex mu;
};

// the "branches" member of a small JSON object, if any
int branches_from_json(const char* js) {
    if (!js) return 0;
    const char* k = std::strstr(js, "\"branches\"");
    if (!k) return 0;
    k = std::strchr(k + 10, ':');
    if (!k) return 0;
    return std::atoi(k + 1);
}

void destroy_cached(Plan* p) {
    for (auto& c : p->cached) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        c.exec = nullptr;
        c.key.clear();
    }
}

// Issue every field of the batch on its branch, forked from and joined into `s`.
toposzp_status enqueue(Plan* p, bool compress, const void* const* a, void* const* b, uint64_t* sizes, void* ws,
                       int32_t* statuses, cudaStream_t s) {
    if (cudaEventRecord(p->ev[0], s) != cudaSuccess) return TOPOSZP_ERR_CUDA;
    for (int k = 0; k < p->branches; k++)
        if (cudaStreamWaitEvent(p->st[k], p->ev[0], 0) != cudaSuccess) return TOPOSZP_ERR_CUDA;
    uint8_t* wsb = static_cast<uint8_t*>(ws);
    for (size_t i = 0; i < p->f.size(); i++) {
        const Field& f = p->f[i];
        cudaStream_t bs = p->st[f.branch];
        void* w = wsb + p->ws_off[f.branch];
        toposzp_status r;
        if (compress)
            r = toposzp_compress(static_cast<const float*>(a[i]), f.ndim, f.dims, f.mode, f.eb, &p->params, b[i],
                                 f.bound, sizes + i, w, f.ws_c, statuses + i, bs);
        else
            r = toposzp_decompress(a[i], f.bound, static_cast<float*>(b[i]), f.n, w, f.ws_d, statuses + i, bs);
        if (r != TOPOSZP_OK) return r;
    }
    for (int k = 0; k < p->branches; k++) {
        if (cudaEventRecord(p->ev[1 + k], p->st[k]) != cudaSuccess) return TOPOSZP_ERR_CUDA;
        if (cudaStreamWaitEvent(s, p->ev[1 + k], 0) != cudaSuccess) return TOPOSZP_ERR_CUDA;
    }
    return TOPOSZP_OK;
}

toposzp_status run(Plan* p, bool compress, const void* const* a, void* const* b, uint64_t* sizes, void* ws,
                   uint64_t ws_bytes, int32_t* statuses, cudaStream_t s) {
    if (!p || !a || !b || !ws || !statuses || (compress && !sizes)) return TOPOSZP_ERR_INVALID_ARG;
    if (ws_bytes < p->ws_bytes) return TOPOSZP_ERR_BUFFER_TOO_SMALL;
    // the test hook would be baked into a captured graph: refuse while it is set
    if (!compress && tsz::test_hold_active()) return TOPOSZP_ERR_INVALID_ARG;
    const size_t nf = p->f.size();
    for (size_t i = 0; i < nf; i++)
        if (!a[i] || !b[i]) return TOPOSZP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(p->mu);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return TOPOSZP_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone)   // inside the caller's capture: plain launches
        return enqueue(p, compress, a, b, sizes, ws, statuses, s);
    // key: every pointer the launches bake in
    std::vector<const void*> key;
    key.reserve(2 * nf + 3);
    for (size_t i = 0; i < nf; i++) {
        key.push_back(a[i]);
        key.push_back(b[i]);
    }
    key.push_back(sizes);
    key.push_back(ws);
    key.push_back(statuses);
    auto& c = p->cached[compress ? 0 : 1];
    if (!c.exec || c.key != key) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        c.exec = nullptr;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TOPOSZP_ERR_CUDA;
        const toposzp_status r = enqueue(p, compress, a, b, sizes, ws, statuses, p->cap);
        const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (r != TOPOSZP_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return TOPOSZP_ERR_CUDA;
        const cudaError_t ie = cudaGraphInstantiate(&c.exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            c.exec = nullptr;
            return TOPOSZP_ERR_CUDA;
        }
        c.key = key;
    }
    return cudaGraphLaunch(c.exec, s) == cudaSuccess ? TOPOSZP_OK : TOPOSZP_ERR_CUDA;
}

}  // namespace

extern "C" {

toposzp_status toposzp_batch_plan_create(int nfields, const int* ndims, const uint64_t* dims3,
                                         const toposzp_eb_mode* modes, const double* ebs,
                                         const toposzp_params* params, const char* tune_json, void** plan) {
    if (!plan || nfields <= 0 || !ndims || !dims3 || !modes || !ebs) return TOPOSZP_ERR_INVALID_ARG;
    *plan = nullptr;
    Plan* p = new (std::nothrow) Plan();
    if (!p) return TOPOSZP_ERR_CUDA;
    if (params) p->params = *params;
    else toposzp_default_params(&p->params);
    p->f.resize(nfields);
    for (int i = 0; i < nfields; i++) {
        Field& f = p->f[i];
        f.ndim = ndims[i];
        for (int d = 0; d < 3; d++) f.dims[d] = dims3[3 * i + d];
        if (f.ndim == 2) f.dims[2] = 1;
        f.mode = modes[i];
        f.eb = ebs[i];
        if ((f.ndim != 2 && f.ndim != 3) || !(f.eb > 0.0) || (f.mode != TOPOSZP_EB_ABS && f.mode != TOPOSZP_EB_REL)) {
            delete p;
            return TOPOSZP_ERR_INVALID_ARG;
        }
        f.n = f.dims[0] * f.dims[1] * f.dims[2];
        f.ws_c = toposzp_compress_workspace_size(f.ndim, f.dims);
        f.ws_d = toposzp_decompress_workspace_size(f.ndim, f.dims);
        f.bound = toposzp_compress_bound(f.ndim, f.dims);
        if (!f.n || !f.ws_c || !f.ws_d || !f.bound) {
            delete p;
            return TOPOSZP_ERR_INVALID_ARG;
        }
    }
    int br = branches_from_json(tune_json);
    if (br <= 0) br = 8;
    p->branches = std::max(1, std::min(br, nfields));
    // longest first onto the least-loaded branch
    std::vector<int> order(nfields);
    for (int i = 0; i < nfields; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return p->f[x].n > p->f[y].n; });
    std::vector<uint64_t> load(p->branches, 0), need(p->branches, 0);
    for (int i : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        p->f[i].branch = b;
        load[b] += p->f[i].n;
        need[b] = std::max(need[b], std::max(p->f[i].ws_c, p->f[i].ws_d));
    }
    p->ws_off.resize(p->branches);
    for (int b = 0; b < p->branches; b++) {
        p->ws_off[b] = p->ws_bytes;
        p->ws_bytes += up(need[b]);
    }
    p->st.resize(p->branches, nullptr);
    p->ev.resize(1 + p->branches, nullptr);
    bool ok = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b < p->branches; b++) ok = cudaStreamCreateWithFlags(&p->st[b], cudaStreamNonBlocking) == cudaSuccess;
    for (size_t e = 0; ok && e < p->ev.size(); e++) ok = cudaEventCreateWithFlags(&p->ev[e], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        toposzp_batch_plan_destroy(p);
        return TOPOSZP_ERR_CUDA;
    }
    *plan = p;
    return TOPOSZP_OK;
}

uint64_t toposzp_batch_workspace_size(const void* plan) {
    return plan ? static_cast<const Plan*>(plan)->ws_bytes : 0;
}

int toposzp_batch_branches(const void* plan) {
    return plan ? static_cast<const Plan*>(plan)->branches : 0;
}

toposzp_status toposzp_batch_compress(void* plan, const float* const* fields, void* const* outs, uint64_t* out_sizes,
                                      void* workspace, uint64_t ws_bytes, int32_t* statuses, toposzp_stream stream) {
    return run(static_cast<Plan*>(plan), true, reinterpret_cast<const void* const*>(fields), outs, out_sizes,
               workspace, ws_bytes, statuses, reinterpret_cast<cudaStream_t>(stream));
}

toposzp_status toposzp_batch_decompress(void* plan, const void* const* ins, float* const* outs, void* workspace,
                                        uint64_t ws_bytes, int32_t* statuses, toposzp_stream stream) {
    return run(static_cast<Plan*>(plan), false, ins, reinterpret_cast<void* const*>(outs), nullptr, workspace,
               ws_bytes, statuses, reinterpret_cast<cudaStream_t>(stream));
}

void toposzp_batch_plan_destroy(void* plan) {
    Plan* p = static_cast<Plan*>(plan);
    if (!p) return;
    destroy_cached(p);
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : p->st)
        if (s) cudaStreamDestroy(s);
    if (p->cap) cudaStreamDestroy(p->cap);
    delete p;
}

}  // extern "C"
