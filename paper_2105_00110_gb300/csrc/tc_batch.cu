// Batches: many independent graphs in one build and one set of persistent
// launches.
//
// A batch is the disjoint union of its graphs: graph k's vertices are
// shifted by voff[k] = Σ_{j<k} n_j.  With no edge between graphs, every
// triangle, count, flag and numerator of the union is that of its own graph
// (Definition 1 only looks at a vertex's neighbourhood); only the
// denominator 3△(G_k) is per graph, and it equals Σ_{v ∈ G_k} △(v).  So the
// union goes through the single-graph build and count unchanged, a
// segmented sum gives each graph's 3△(G_k), and the gather divides every
// vertex by its own graph's value.
//
// tc_batch_run makes no host synchronisation and no allocation, so a run can
// be captured into a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "tc_internal.cuh"

struct tc_batch {
    tc_graph* g = nullptr;               // the disjoint union
    int64_t num_graphs = 0;
    int64_t* voff = nullptr;             // [G+1] vertex offsets (device)
    int64_t* eoff = nullptr;             // [G+1] canonical-edge offsets (device)
    int32_t* rank_graph = nullptr;       // [n] graph of each rank
    unsigned long long* sums = nullptr;  // [G] Σ△(v) = 3△(G_k)
    std::vector<int64_t> h_voff, h_eoff;
};

namespace tcx {
namespace {

typedef unsigned long long ull;

inline int blocks(int64_t items) {
    int64_t b = (items + 255) / 256, cap = (int64_t)sm_count() * 16;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

// Pairs of graph k (pairs [poff[k], poff[k+1])) -> union labels; an id
// outside [0, n_k) sets the error word.
template <typename T>
__global__ void k_shift_pairs(const T* __restrict__ src, const T* __restrict__ dst, int64_t np,
                              const int64_t* __restrict__ poff, const int64_t* __restrict__ voff,
                              int64_t G, int32_t* __restrict__ gs, int32_t* __restrict__ gd,
                              unsigned int* __restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = G;   // last k with poff[k] <= i
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (poff[mid] <= i) lo = mid; else hi = mid;
        }
        const int64_t nk = voff[lo + 1] - voff[lo];
        const int64_t a = (int64_t)src[i], b = (int64_t)dst[i];
        if (a < 0 || b < 0 || a >= nk || b >= nk) {
            atomicOr(err, 1u);
            gs[i] = gd[i] = 0;
        } else {
            gs[i] = (int32_t)(voff[lo] + a);
            gd[i] = (int32_t)(voff[lo] + b);
        }
    }
}

// graph of every rank (through its union label)
__global__ void k_rank_graph(const int32_t* __restrict__ perm, int64_t n, const int64_t* __restrict__ voff,
                             int64_t G, int32_t* __restrict__ rg) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = perm[r];
        int64_t lo = 0, hi = G;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (voff[mid] <= v) lo = mid; else hi = mid;
        }
        rg[r] = (int32_t)lo;
    }
}

// first canonical edge of every graph (edges are sorted by union label)
__global__ void k_edge_offsets(const int32_t* __restrict__ eu, int64_t m, const int64_t* __restrict__ voff,
                               int64_t G, int64_t* __restrict__ eoff) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= G;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = voff[k];
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)eu[mid] < x) lo = mid + 1; else hi = mid;
        }
        eoff[k] = lo;
    }
}

__global__ void k_totals(const ull* __restrict__ sums, int64_t G, ull* __restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < G;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = sums[k] / 3;
}

void free_batch(tc_batch* b, cudaStream_t s) {
    if (b->g) {
        b->g->rank_graph = nullptr;
        b->g->den_graph = nullptr;
        free_graph_memory(b->g);
        delete b->g;
        b->g = nullptr;
    }
    dfree(b->voff, s);
    dfree(b->eoff, s);
    dfree(b->rank_graph, s);
    dfree(b->sums, s);
}

tc_status build_batch(tc_batch* b, const void* src, const void* dst, const int64_t* h_poff,
                      const int64_t* h_nv, int64_t G, uint32_t flags, cudaStream_t s) {
    b->num_graphs = G;
    b->h_voff.assign(G + 1, 0);
    for (int64_t k = 0; k < G; ++k) {
        if (h_nv[k] < 0 || h_poff[k + 1] < h_poff[k]) return TC_ERR_INVALID_ARG;
        b->h_voff[k + 1] = b->h_voff[k] + h_nv[k];
    }
    if (h_poff[0] != 0) return TC_ERR_INVALID_ARG;
    const int64_t n = b->h_voff[G], np = h_poff[G];
    if (n > INT32_MAX) return TC_ERR_INVALID_ARG;
    if (np > 0 && (!src || !dst)) return TC_ERR_INVALID_ARG;
    const bool i32 = (flags & TC_IDS_INT32) != 0;
    const size_t idb = i32 ? 4 : 8;

    std::vector<void*> tmp;
    auto cleanup = [&] {
        for (void* q : tmp) dfree(q, s);
    };
#define B_TRY(x)                 \
    do {                         \
        tc_status _s = (x);      \
        if (_s < 0) {            \
            cleanup();           \
            return _s;           \
        }                        \
    } while (0)
    auto get = [&](void** q, size_t bytes) -> tc_status {
        tc_status st = dalloc(q, bytes, s);
        if (st == TC_OK) tmp.push_back(*q);
        return st;
    };
    B_TRY(dalloc((void**)&b->voff, (G + 1) * 8, s));
    B_TRY(dalloc((void**)&b->eoff, (G + 1) * 8, s));
    B_TRY(dalloc((void**)&b->sums, (G + 1) * 8, s));
    B_TRY(from_cuda(cudaMemcpyAsync(b->voff, b->h_voff.data(), (G + 1) * 8, cudaMemcpyHostToDevice, s)));
    int64_t* poff = nullptr;
    B_TRY(get((void**)&poff, (G + 1) * 8));
    B_TRY(from_cuda(cudaMemcpyAsync(poff, h_poff, (G + 1) * 8, cudaMemcpyHostToDevice, s)));
    const void *dsrc = src, *ddst = dst;
    if (!(flags & TC_IN_DEVICE) && np > 0) {
        void *a = nullptr, *c = nullptr;
        B_TRY(get(&a, np * idb));
        B_TRY(get(&c, np * idb));
        B_TRY(from_cuda(cudaMemcpyAsync(a, src, np * idb, cudaMemcpyHostToDevice, s)));
        B_TRY(from_cuda(cudaMemcpyAsync(c, dst, np * idb, cudaMemcpyHostToDevice, s)));
        dsrc = a;
        ddst = c;
    }
    int32_t *gs = nullptr, *gd = nullptr;
    unsigned int* err = nullptr;
    B_TRY(get((void**)&gs, (np + 1) * 4));
    B_TRY(get((void**)&gd, (np + 1) * 4));
    B_TRY(get((void**)&err, 4));
    B_TRY(from_cuda(cudaMemsetAsync(err, 0, 4, s)));
    if (np > 0) {
        launch_scope ls("batch_shift_pairs", s);
        if (i32)
            k_shift_pairs<int32_t><<<blocks(np), 256, 0, s>>>((const int32_t*)dsrc, (const int32_t*)ddst, np,
                                                              poff, b->voff, G, gs, gd, err);
        else
            k_shift_pairs<int64_t><<<blocks(np), 256, 0, s>>>((const int64_t*)dsrc, (const int64_t*)ddst, np,
                                                              poff, b->voff, G, gs, gd, err);
        B_TRY(from_cuda(cudaGetLastError()));
    }
    unsigned int h_err = 0;
    B_TRY(from_cuda(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s)));
    B_TRY(from_cuda(cudaStreamSynchronize(s)));
    if (h_err) {
        cleanup();
        return TC_ERR_INVALID_ARG;
    }
    b->g = new (std::nothrow) tc_graph();
    if (!b->g) {
        cleanup();
        return TC_ERR_OUT_OF_MEMORY;
    }
    cudaGetDevice(&b->g->device);
    B_TRY(build_graph(b->g, gs, gd, np, n, TC_IN_DEVICE | TC_IDS_INT32 | TC_BUILD_NO_CORE, s));
    tc_graph* g = b->g;
    B_TRY(dalloc((void**)&b->rank_graph, (n + 1) * 4, s));
    if (n > 0) {
        launch_scope ls("batch_rank_graph", s);
        k_rank_graph<<<blocks(n), 256, 0, s>>>(g->perm, n, b->voff, G, b->rank_graph);
        B_TRY(from_cuda(cudaGetLastError()));
    }
    {
        launch_scope ls("batch_edge_offsets", s);
        k_edge_offsets<<<blocks(G + 1), 256, 0, s>>>(g->edge_u, g->m, b->voff, G, b->eoff);
        B_TRY(from_cuda(cudaGetLastError()));
    }
    b->h_eoff.assign(G + 1, 0);
    B_TRY(from_cuda(cudaMemcpyAsync(b->h_eoff.data(), b->eoff, (G + 1) * 8, cudaMemcpyDeviceToHost, s)));
    g->rank_graph = b->rank_graph;
    g->den_graph = b->sums;
    B_TRY(from_cuda(cudaStreamSynchronize(s)));
    cleanup();
    return TC_OK;
#undef B_TRY
}

}  // namespace

tc_status run_batch(tc_batch* b, uint64_t* d_tri, uint8_t* d_flag, uint64_t* d_numer, double* d_tc,
                    uint64_t* d_totals, cudaStream_t s) {
    tc_graph* g = b->g;
    g->stream = s;
    TC_TRY(run_count(g, s));
    TC_CUDA(cudaMemsetAsync(b->sums, 0, (b->num_graphs + 1) * 8, s));
    TC_TRY(run_graph_sums(g, b->rank_graph, b->sums, s));
    if (d_numer || d_tc) TC_TRY(run_centrality(g, d_numer, d_tc, s));
    if (d_tri) TC_TRY(export_tri(g, d_tri, s));
    if (d_flag) TC_TRY(export_flags(g, d_flag, s));
    if (d_totals && b->num_graphs > 0) {
        launch_scope ls("batch_totals", s);
        k_totals<<<blocks(b->num_graphs), 256, 0, s>>>(b->sums, b->num_graphs, (ull*)d_totals);
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}

}  // namespace tcx

using namespace tcx;

extern "C" {

tc_status tc_batch_build(const void* src, const void* dst, const int64_t* h_pair_offsets,
                         const int64_t* h_num_vertices, int64_t num_graphs, uint32_t flags,
                         tc_stream stream, tc_batch** out) {
    tcx::nvtx_range nr("tc_batch_build");
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (num_graphs < 0 || (num_graphs > 0 && (!h_pair_offsets || !h_num_vertices)))
        return TC_ERR_INVALID_ARG;
    if (flags & ~(TC_IN_DEVICE | TC_IDS_INT32)) return TC_ERR_INVALID_ARG;
    const int64_t zero = 0;
    if (num_graphs == 0) h_pair_offsets = &zero;
    tc_batch* b = new (std::nothrow) tc_batch();
    if (!b) return TC_ERR_OUT_OF_MEMORY;
    cudaStream_t s = (cudaStream_t)stream;
    tc_status st;
    try {
        st = build_batch(b, src, dst, h_pair_offsets, h_num_vertices, num_graphs, flags, s);
    } catch (...) {
        st = TC_ERR_OUT_OF_MEMORY;
    }
    if (st >= 0) st = [&]() -> tc_status {
        TC_DEBUG_COLLECT(s);   // bounds-checked builds only
        return TC_OK;
    }();
    if (st < 0) {
        free_batch(b, s);
        cudaStreamSynchronize(s);
        delete b;
        return st;
    }
    *out = b;
    return TC_OK;
}

tc_status tc_batch_run(tc_batch* b, uint64_t* d_tri, uint8_t* d_edge_flag, uint64_t* d_numer, double* d_tc,
                       uint64_t* d_tri_totals, tc_stream stream) {
    tcx::nvtx_range nr("tc_batch_run");
    if (!b) return TC_ERR_INVALID_ARG;
    TC_TRY(run_batch(b, d_tri, d_edge_flag, d_numer, d_tc, d_tri_totals, (cudaStream_t)stream));
    TC_DEBUG_COLLECT((cudaStream_t)stream);   // bounds-checked builds only: synchronises
    return TC_OK;
}

tc_status tc_batch_info(const tc_batch* b, int64_t* num_graphs, int64_t* num_vertices, int64_t* num_edges,
                        int64_t* h_vertex_offsets, int64_t* h_edge_offsets) {
    if (!b) return TC_ERR_INVALID_ARG;
    if (num_graphs) *num_graphs = b->num_graphs;
    if (num_vertices) *num_vertices = b->g->n;
    if (num_edges) *num_edges = b->g->m;
    if (h_vertex_offsets) std::memcpy(h_vertex_offsets, b->h_voff.data(), (b->num_graphs + 1) * 8);
    if (h_edge_offsets) std::memcpy(h_edge_offsets, b->h_eoff.data(), (b->num_graphs + 1) * 8);
    return TC_OK;
}

tc_status tc_batch_copy_edges(const tc_batch* b, int32_t* d_u, int32_t* d_v, tc_stream stream) {
    if (!b) return TC_ERR_INVALID_ARG;
    return tc_copy_edges(b->g, d_u, d_v, stream);
}

tc_status tc_batch_get_stats(const tc_batch* b, tc_graph_stats* out) {
    if (!b) return TC_ERR_INVALID_ARG;
    return tc_get_stats(b->g, out);
}

tc_status tc_batch_autotune(tc_batch* b, int reps, tc_stream stream) {
    if (!b || reps < 1) return TC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    tc_graph* g = b->g;
    // candidate planner settings: when a vertex is heavy enough for a CTA
    // item, and how much work one CTA or warp item carries
    const tc_plan_params cands[] = {
        {4096, 4194304, 32768}, {4096, 65536, 16384}, {1024, 65536, 16384}, {16384, 65536, 16384},
        {4096, 32768, 8192},    {4096, 131072, 32768}, {1024, 32768, 4096},  {4096, 65536, 65536},
    };
    cudaEvent_t e0, e1;
    TC_CUDA(cudaEventCreate(&e0));
    TC_CUDA(cudaEventCreate(&e1));
    float best = 3.4e38f;
    tc_plan_params best_p = g->params;
    tc_status st = TC_OK;
    for (const tc_plan_params& c : cands) {
        g->params = c;
        g->params.thread_work = best_p.thread_work;   // not one of the tuned settings
        g->params_version += 1;
        st = run_count(g, s);   // re-plans for the new parameters, then warms up
        if (st < 0) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st >= 0; ++r) st = run_count(g, s);
        cudaEventRecord(e1, s);
        if (st < 0) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = TC_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_p = g->params;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->params = best_p;
    g->params_version += 1;
    if (st >= 0) st = make_plan(g, g->strategy, s);
    return st;
}

tc_status tc_batch_get_params(const tc_batch* b, int64_t* out3) {
    if (!b || !out3) return TC_ERR_INVALID_ARG;
    out3[0] = b->g->params.cta_min_work;
    out3[1] = b->g->params.cta_chunk;
    out3[2] = b->g->params.warp_chunk;
    return TC_OK;
}

void tc_batch_free(tc_batch* b) {
    if (!b) return;
    cudaStream_t s = b->g ? b->g->stream : nullptr;
    free_batch(b, s);
    cudaStreamSynchronize(s);
    delete b;
}

}  // extern "C"
