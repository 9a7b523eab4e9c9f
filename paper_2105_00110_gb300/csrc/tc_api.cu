// C-ABI entry points, status strings, allocation and launch accounting.
#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "tc_internal.cuh"

namespace tcx {

tc_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TC_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return TC_ERR_OUT_OF_MEMORY;
    }
    return TC_ERR_CUDA;
}

namespace {
std::once_flag g_pool_once;
std::atomic<long long> g_launches{0};
// failure injection and accounting of the device allocations (testing aid)
std::atomic<long long> g_fail_in{-1};     // allocations left before the injected failure; -1 off
std::atomic<long long> g_allocs{0};       // device allocations requested since load
std::atomic<long long> g_live{0};         // device allocations currently held

struct timing_rec {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<timing_rec> g_pending;      // launch-bracketing events not yet read
std::vector<tc_kernel_time> g_totals;   // accumulated per name
std::vector<cudaEvent_t> g_free_events;
thread_local cudaEvent_t t_start = nullptr;

cudaEvent_t take_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void accumulate(const char* name, float ms) {
    for (auto& t : g_totals)
        if (std::strncmp(t.name, name, sizeof(t.name)) == 0) {
            t.launches += 1;
            t.total_ms += ms;
            return;
        }
    tc_kernel_time k{};
    std::strncpy(k.name, name, sizeof(k.name) - 1);
    k.launches = 1;
    k.total_ms = ms;
    g_totals.push_back(k);
}

void drain_locked() {
    for (auto& r : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
            accumulate(r.name, ms);
        g_free_events.push_back(r.a);
        g_free_events.push_back(r.b);
    }
    g_pending.clear();
}
}  // namespace

#ifdef TC_DEBUG_BOUNDS
namespace {
std::mutex& dbg_mu() {
    static std::mutex m;
    return m;
}
std::vector<unsigned (*)()>& dbg_readers() {
    static std::vector<unsigned (*)()> v;
    return v;
}
std::atomic<long long> g_dbg_line{0};
}  // namespace

void dbg_register(unsigned (*take)()) {
    std::lock_guard<std::mutex> lk(dbg_mu());
    dbg_readers().push_back(take);
}

tc_status dbg_collect() {
    std::lock_guard<std::mutex> lk(dbg_mu());
    unsigned line = 0;
    for (auto take : dbg_readers()) {
        const unsigned v = take();
        if (v && !line) line = v;
    }
    if (line) g_dbg_line.store(line);
    return line ? TC_ERR_BOUNDS : TC_OK;
}
#endif

int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

tc_status dalloc(void** p, size_t bytes, cudaStream_t s) {
    std::call_once(g_pool_once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            // keep freed blocks cached in this process so that repeated
            // builds do not return memory to the driver in between
            uint64_t threshold = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
        }
    });
    *p = nullptr;
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    // an armed injected failure: the allocation that takes the count to -1
    // fails as a device out-of-memory would, once
    long long k = g_fail_in.load();
    while (k >= 0 && !g_fail_in.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) return TC_ERR_OUT_OF_MEMORY;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return from_cuda(e);
    }
    g_live.fetch_add(1, std::memory_order_relaxed);
    return TC_OK;
}

void dfree(void* p, cudaStream_t s) {
    if (p) {
        cudaFreeAsync(p, s);
        g_live.fetch_sub(1, std::memory_order_relaxed);
    }
}

void add_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int64_t library_kernels(const char* site, int64_t size, int64_t bits,
                        const std::function<cudaError_t(cudaStream_t)>& call) {
    static std::mutex mu;
    static std::map<std::tuple<std::string, int64_t, int64_t>, int64_t> known;
    const auto key = std::make_tuple(std::string(site), size, bits);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = known.find(key);
        if (it != known.end()) return it->second;
    }
    int64_t kernels = 1;   // if the count cannot be taken, the call counts once
    cudaStream_t probe = nullptr;
    if (cudaStreamCreateWithFlags(&probe, cudaStreamNonBlocking) == cudaSuccess) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(probe, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t e = call(probe);
            if (cudaStreamEndCapture(probe, &graph) == cudaSuccess && e == cudaSuccess && graph) {
                size_t nn = 0;
                if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
                    std::vector<cudaGraphNode_t> nodes(nn);
                    if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess) {
                        int64_t k = 0;
                        for (size_t i = 0; i < nn; ++i) {
                            cudaGraphNodeType t;
                            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
                        }
                        kernels = k;
                    }
                }
            }
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();   // a failed capture leaves no error behind for the caller
        cudaStreamDestroy(probe);
    }
    std::lock_guard<std::mutex> lk(mu);
    known[key] = kernels;
    return kernels;
}

void note_launch(const char* name, cudaStream_t s, int phase, bool counts) {
    if (phase == 0) {
        if (counts) g_launches.fetch_add(1, std::memory_order_relaxed);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (g_prof_on) {
            t_start = take_event();
            cudaEventRecord(t_start, s);
        } else {
            t_start = nullptr;
        }
    } else {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (g_prof_on && t_start) {
            cudaEvent_t b = take_event();
            cudaEventRecord(b, s);
            g_pending.push_back({name, t_start, b});
            t_start = nullptr;
        }
    }
}

}  // namespace tcx

using namespace tcx;

extern "C" {

const char* tc_status_str(tc_status s) {
    switch (s) {
        case TC_OK: return "ok";
        case TC_NO_TRIANGLES: return "graph has no triangles (TC undefined, NaN)";
        case TC_ERR_INVALID_ARG: return "invalid argument";
        case TC_ERR_OUT_OF_MEMORY: return "out of memory";
        case TC_ERR_CUDA: return "CUDA error";
        case TC_ERR_OVERFLOW: return "3 * triangle count overflows 64 bits";
        case TC_ERR_TIMEOUT: return "device wait timed out";
        case TC_ERR_STATE: return "call order violated";
        case TC_ERR_BOUNDS: return "a device bounds check failed (bounds-checked build)";
    }
    return "unknown status";
}

tc_status tc_build_csr(const void* src, const void* dst, int64_t num_pairs, int64_t n,
                       uint32_t flags, tc_stream stream, tc_graph** out) {
    nvtx_range nr("tc_build_csr");
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (num_pairs < 0 || n < 0 || n > INT32_MAX) return TC_ERR_INVALID_ARG;
    if (num_pairs > 0 && (!src || !dst)) return TC_ERR_INVALID_ARG;
    if (flags & ~(TC_IN_DEVICE | TC_IDS_INT32)) return TC_ERR_INVALID_ARG;
    tc_graph* g = new (std::nothrow) tc_graph();
    if (!g) return TC_ERR_OUT_OF_MEMORY;
    cudaGetDevice(&g->device);
    tc_status st;
    try {
        st = build_graph(g, src, dst, num_pairs, n, flags, (cudaStream_t)stream);
    } catch (...) {
        st = TC_ERR_CUDA;
    }
    if (st >= 0) st = [&]() -> tc_status {
        TC_DEBUG_COLLECT((cudaStream_t)stream);   // bounds-checked builds only
        return TC_OK;
    }();
    if (st < 0) {
        free_graph_memory(g);
        cudaStreamSynchronize((cudaStream_t)stream);
        delete g;
        return st;
    }
    *out = g;
    return TC_OK;
}

tc_status tc_count(tc_graph* g, uint64_t* d_tri, uint8_t* d_edge_flag, uint64_t* h_tri_total,
                   tc_stream stream) {
    nvtx_range nr("tc_count");
    if (!g) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    g->counted = 0;
    TC_TRY(run_count(g, s));
    if (d_tri) TC_TRY(export_tri(g, d_tri, s));
    if (d_edge_flag) TC_TRY(export_flags(g, d_edge_flag, s));
    unsigned long long total = 0;
    TC_CUDA(cudaMemcpyAsync(&total, g->counters, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    TC_DEBUG_COLLECT(s);
    g->total = total;
    g->counted = 1;
    if (h_tri_total) *h_tri_total = total;
    return total == 0 ? TC_NO_TRIANGLES : TC_OK;
}

tc_status tc_edge_triangles(tc_graph* g, uint64_t* d_tri, uint32_t* d_edge_tri, uint64_t* h_tri_total,
                            tc_stream stream) {
    nvtx_range nr("tc_edge_triangles");
    if (!g) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    g->counted = 0;
    TC_TRY(run_count(g, s, true));
    if (d_tri) TC_TRY(export_tri(g, d_tri, s));
    if (d_edge_tri) TC_TRY(export_edge_counts(g, d_edge_tri, s));
    unsigned long long total = 0;
    TC_CUDA(cudaMemcpyAsync(&total, g->counters, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    TC_DEBUG_COLLECT(s);
    g->total = total;
    g->counted = 1;
    if (h_tri_total) *h_tri_total = total;
    return total == 0 ? TC_NO_TRIANGLES : TC_OK;
}

tc_status tc_count_shard(tc_graph* g, int shard, int num_shards, uint64_t* d_tri, uint8_t* d_edge_flag,
                         uint64_t* h_tri_partial, tc_stream stream) {
    nvtx_range nr("tc_count_shard");
    if (!g || num_shards < 1 || shard < 0 || shard >= num_shards) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    g->counted = 0;   // partial counts: tc_centrality needs tc_load_counts first
    TC_TRY(run_count(g, s, false, shard, num_shards));
    if (d_tri) TC_TRY(export_tri(g, d_tri, s));
    if (d_edge_flag) TC_TRY(export_flags(g, d_edge_flag, s));
    unsigned long long part = 0;
    TC_CUDA(cudaMemcpyAsync(&part, g->counters, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    TC_DEBUG_COLLECT(s);
    if (h_tri_partial) *h_tri_partial = part;
    return TC_OK;
}

tc_status tc_load_counts(tc_graph* g, const uint64_t* d_tri, const uint8_t* d_edge_flag, uint64_t* h_tri_total,
                         tc_stream stream) {
    nvtx_range nr("tc_load_counts");
    if (!g || (g->n > 0 && !d_tri) || (g->m > 0 && !d_edge_flag)) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    g->counted = 0;
    TC_TRY(import_counts(g, d_tri, d_edge_flag, s));
    unsigned long long sum = 0;
    TC_CUDA(cudaMemcpyAsync(&sum, g->counters, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    TC_DEBUG_COLLECT(s);
    if (sum % 3 != 0) return TC_ERR_INVALID_ARG;   // Σ △(v) = 3△(G) for any graph
    g->total = sum / 3;
    TC_CUDA(cudaMemcpyAsync(g->counters, &g->total, 8, cudaMemcpyHostToDevice, s));
    TC_CUDA(cudaStreamSynchronize(s));
    g->counted = 1;
    if (h_tri_total) *h_tri_total = g->total;
    return g->total == 0 ? TC_NO_TRIANGLES : TC_OK;
}

tc_status tc_centrality(tc_graph* g, uint64_t* d_numer, double* d_tc, uint64_t* h_den,
                        tc_stream stream) {
    nvtx_range nr("tc_centrality");
    if (!g) return TC_ERR_INVALID_ARG;
    if (!g->counted) return TC_ERR_STATE;
    if (g->total > UINT64_MAX / 3) return TC_ERR_OVERFLOW;
    g->stream = (cudaStream_t)stream;
    TC_TRY(run_centrality(g, d_numer, d_tc, (cudaStream_t)stream));
    TC_DEBUG_COLLECT((cudaStream_t)stream);   // bounds-checked builds only: synchronises
    if (h_den) *h_den = 3ull * g->total;
    return g->total == 0 ? TC_NO_TRIANGLES : TC_OK;
}

tc_status tc_divide(const uint64_t* d_numer, int64_t n, uint64_t den, double* d_tc, tc_stream stream) {
    if (n < 0 || (n > 0 && (!d_numer || !d_tc))) return TC_ERR_INVALID_ARG;
    return run_divide(d_numer, n, den, d_tc, (cudaStream_t)stream);
}

tc_status tc_graph_info(const tc_graph* g, int64_t* n, int64_t* m, const int32_t** d_edge_u,
                        const int32_t** d_edge_v) {
    if (!g) return TC_ERR_INVALID_ARG;
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (d_edge_u) *d_edge_u = g->edge_u;
    if (d_edge_v) *d_edge_v = g->edge_v;
    return TC_OK;
}

tc_status tc_copy_edges(const tc_graph* g, int32_t* d_u, int32_t* d_v, tc_stream stream) {
    if (!g) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->m > 0 && d_u) TC_CUDA(cudaMemcpyAsync(d_u, g->edge_u, g->m * 4, cudaMemcpyDeviceToDevice, s));
    if (g->m > 0 && d_v) TC_CUDA(cudaMemcpyAsync(d_v, g->edge_v, g->m * 4, cudaMemcpyDeviceToDevice, s));
    return TC_OK;
}

tc_status tc_get_stats(const tc_graph* g, tc_graph_stats* out) {
    if (!g || !out) return TC_ERR_INVALID_ARG;
    *out = g->stats;
    out->core_vertices = g->core_c;
    return TC_OK;
}

tc_status tc_set_plan_params(tc_graph* g, const int64_t* params3) {
    if (!g || !params3 || params3[0] < 0 || params3[1] < 1 || params3[2] < 1) return TC_ERR_INVALID_ARG;
    g->params.cta_min_work = params3[0];
    g->params.cta_chunk = params3[1];
    g->params.warp_chunk = params3[2];
    g->params_version += 1;   // the next count re-plans
    return TC_OK;
}

tc_status tc_get_plan_params(const tc_graph* g, int64_t* out3) {
    if (!g || !out3) return TC_ERR_INVALID_ARG;
    out3[0] = g->params.cta_min_work;
    out3[1] = g->params.cta_chunk;
    out3[2] = g->params.warp_chunk;
    return TC_OK;
}

tc_status tc_set_strategy(tc_graph* g, int strategy) {
    if (!g || strategy < TC_STRATEGY_AUTO || strategy > TC_STRATEGY_GLOBAL) return TC_ERR_INVALID_ARG;
    g->strategy = strategy;
    return TC_OK;
}

tc_status tc_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return TC_OK;
}

tc_status tc_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    g_totals.clear();
    return TC_OK;
}

tc_status tc_profile_read(tc_kernel_time* out, int cap, int* count) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    int k = 0;
    for (auto& t : g_totals) {
        if (out && k < cap) out[k] = t;
        ++k;
    }
    if (count) *count = k;
    return TC_OK;
}

int64_t tc_launch_count(void) { return (int64_t)g_launches.load(); }

int tc_debug_bounds_build(void) {
#ifdef TC_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

int64_t tc_debug_bounds_line(void) {
#ifdef TC_DEBUG_BOUNDS
    return (int64_t)tcx::g_dbg_line.load();
#else
    return 0;
#endif
}

tc_status tc_debug_fail_allocation(int64_t k) {
    g_fail_in.store(k < 0 ? -1 : (long long)k);
    return TC_OK;
}

int64_t tc_debug_allocations(void) { return (int64_t)g_allocs.load(); }

int64_t tc_debug_live_allocations(void) { return (int64_t)g_live.load(); }

void tc_graph_free(tc_graph* g) {
    if (!g) return;
    free_graph_memory(g);
    cudaStreamSynchronize(g->stream);
    delete g;
}

}  // extern "C"
