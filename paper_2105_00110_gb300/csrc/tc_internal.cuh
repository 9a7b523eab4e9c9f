// Internal declarations of the GB300 triangle-centrality library.
//
// Device layout of a built graph (all in the degree-ordered label space
// "rank": rank r is the r-th vertex in the order π of section "Notation",
// ascending degree, ties by caller label):
//
//   row_ptr[n+1]  int64   symmetric CSR offsets, row r = rank r
//   col[2m]       int32   neighbour ranks, each row ascending, so row r is
//                         [ N_L(r) | N_H(r) ] with the split at hstart[r]
//   hstart[n]     int64   first position of N_H(r) in row r
//   head[2m]      16 B    for a head entry p = (v, u), u < v (row v's part
//                         [row_ptr, hstart), in no particular order): the
//                         record {u, hrem, twin}: twin = the position of v
//                         inside N_H(u) (row u), hrem = |{w ∈ N_H(u) : w > v}|,
//                         the part of N_H(u) that can close a triangle with
//                         the oriented edge u -> v.  col[] is not written at
//                         head positions; tail positions hold N_H(v) ascending
//   edge_tail[m]  int64   canonical edge e -> its tail position in rank space
//   flag[2m/32]   uint32  one bit per CSR position: the in-a-triangle flag of
//                         each edge, on its tail entry (65 MB at m = 2.6e8,
//                         small enough to stay in L2 while the count runs)
//   perm[n]       int32   rank -> caller label
//   edge_u/v[m]   int32   canonical undirected edges, caller labels, u < v,
//                         sorted by (u, v)
//
// Work items of the count step (the planner's output): an item is a middle
// vertex v and a range [pb, pe) of its head entries (lower neighbours u).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <functional>

#include "tc.h"

#ifndef TC_WARP_CAP
#define TC_WARP_CAP 512          // N_H(v) ids staged per warp item
#endif
#define TC_CTA_THREADS 256

// Item classes of the count step.
enum tc_item_class {
    TC_CLS_BITMAP_S = 0,   // CTA, N_H(v) as a bitmap over its id window, small shared footprint
    TC_CLS_BITMAP_L = 1,   // CTA, bitmap with a large shared footprint
    TC_CLS_WARP = 2,       // warp, N_H(v) as a sorted list (binary search or merge)
    TC_CLS_CTA_LIST = 3,   // CTA, sorted list in shared memory (or global if it does not fit)
    TC_CLS_THREAD = 4,     // one thread per tiny vertex, N_H(v) merged against each stream
    TC_NUM_CLS = 5
};

// A head entry (see the layout above).
struct __align__(16) tc_head {
    int32_t u;
    int32_t hrem;
    int64_t twin;
};

// Planner parameters (tuned per batch by tc_batch_autotune).
#ifndef TC_THREAD_WORK
#define TC_THREAD_WORK 64
#endif
struct tc_plan_params {
    int64_t cta_min_work = 4096;   // W(v) at or above which v may become CTA items
    int64_t cta_chunk = 4194304;   // target wedges per CTA item (each chunk re-stages N_H(v));
                                   // the build sets it from the graph's wedges
    int64_t warp_chunk = 32768;    // target wedges per warp item
    int64_t thread_work = TC_THREAD_WORK;   // head entries + streamed ids at or below which a vertex
                                   // with |N_H(v)| <= 32 is one thread's item (unions of many
                                   // graphs: 128, set by the build)
};

// What a count kernel needs of an item's middle vertex v, in one 16-byte
// load: where N_H(v) starts in the CSR and how long it is (so that staging
// does not wait on two dependent loads of row_ptr and hstart first).
struct tc_item {
    int64_t h0;    // hstart[v]
    int32_t v;
    int32_t hv;    // |N_H(v)|
};

struct tc_plan {
    int strategy = -1;                 // strategy the plan was made for
    int64_t count[TC_NUM_CLS] = {};
    tc_item* d[TC_NUM_CLS] = {};       // middle vertex of each item
    int32_t* nb[TC_NUM_CLS] = {};      // its id window max N_H(v) - v (0 if N_H(v) is empty)
    int64_t* pb[TC_NUM_CLS] = {};      // head-entry range [pb, pe) of the item
    int64_t* pe[TC_NUM_CLS] = {};
    size_t smem[TC_NUM_CLS] = {};      // dynamic shared memory of the class's kernel
    int thread_max_h = 0;              // largest |N_H(v)| of the thread items
};

struct tc_graph {
    int64_t n = 0, m = 0;
    int bits = 1;                // bits needed for a label in [0, n)
    int device = 0;
    cudaStream_t stream = nullptr;
    // canonical (caller labels)
    int32_t* edge_u = nullptr;
    int32_t* edge_v = nullptr;
    int32_t* perm = nullptr;
    // rank space
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    int64_t* hstart = nullptr;
    tc_head* head = nullptr;
    int64_t* edge_tail = nullptr;
    int64_t* work = nullptr;             // [n] W(v) = Σ_{u ∈ N_L(v)} hrem(u, v)
    int64_t band[2] = {0, 0};            // first rank of degree > 32, of degree > 4096
    tc_plan plan;
    // workspace of tc_count / tc_centrality
    unsigned long long* tri = nullptr;   // [n], rank space
    uint32_t* flag = nullptr;            // one bit per CSR position (2m bits), set on tail entries
    uint32_t* ecnt = nullptr;            // [2m] triangles on each tail entry (edge-count mode only)
    uint32_t* tri32 = nullptr;           // [n], rank space: △(v) for the gather's neighbour
                                         // reads, 0xffffffff where △(v) >= 2^32 (then read tri)
    unsigned long long* counters = nullptr;  // [8]: 0 total, 1 warp cursor, 2 cta cursor
    int counted = 0;
    uint64_t total = 0;
    int strategy = TC_STRATEGY_AUTO;
    tc_plan_params params;
    int plan_params_version = 0, params_version = 0;
    tc_graph_stats stats{};
    // dense core: the top core_c ranks, whose mutual triangles the count
    // takes edge by edge from bit-packed core rows (0: none; the head
    // entries whose lower end is in the core then stream nothing)
    int64_t core_c = 0;
    // optional per-graph denominators (batches): rank -> graph, Σ△(v) per graph
    const int32_t* rank_graph = nullptr;
    const unsigned long long* den_graph = nullptr;
};

#define TC_TRY(expr)                                    \
    do {                                                \
        tc_status _st = (expr);                         \
        if (_st < 0) return _st;                        \
    } while (0)

#define TC_CUDA(expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return tcx::from_cuda(_e); \
    } while (0)

#define TC_LAUNCH_CHECK() TC_CUDA(cudaGetLastError())

// ------------------------------------------------------- bounds checks
// Sizes of a built graph's arrays, handed to the kernels whose indices
// come from graph data, for the bounds-checked build.
struct tc_dims {
    int64_t n;    // vertices: tri, numer, perm, hstart (rank space)
    int64_t e2;   // CSR entries (2m): head, ecnt; col holds e2 + 32 (guard ids)
    int64_t fw;   // 32-bit words of the flag bitmap
};

// Bounds-checked builds (-DTC_DEBUG_BOUNDS): TC_IX(i, size) checks an
// index against its array's size.  A failed check records its source line
// in this translation unit's error word and redirects the access to entry
// 0 (every checked array has one), so the kernel never leaves its buffers;
// the entry point then returns TC_ERR_BOUNDS.  No trap, no device assert.
// In other builds TC_IX(i, size) is just i.
#ifdef TC_DEBUG_BOUNDS
static __device__ unsigned int tc_dbg_err_word;
template <class I>
__device__ __forceinline__ I tc_dbg_ix(I i, long long size, int line) {
    if ((unsigned long long)(long long)i >= (unsigned long long)size) {
        atomicCAS(&tc_dbg_err_word, 0u, (unsigned)line);
        return (I)0;
    }
    return i;
}
#define TC_IX(i, size) tc_dbg_ix((i), (long long)(size), __LINE__)
namespace tcx {
// every translation unit registers a reader of its own error word
void dbg_register(unsigned (*take)());
// reads and clears every unit's word: TC_ERR_BOUNDS if one was set
tc_status dbg_collect();
static unsigned dbg_take_here() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, tc_dbg_err_word, sizeof(v)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(tc_dbg_err_word, &z, sizeof(z));
    return v;
}
static const bool tc_dbg_registered = (dbg_register(&dbg_take_here), true);
}  // namespace tcx
#define TC_DEBUG_COLLECT(s)                                   \
    do {                                                      \
        TC_CUDA(cudaStreamSynchronize(s));                    \
        TC_TRY(tcx::dbg_collect());                           \
    } while (0)
#else
#define TC_IX(i, size) (i)
#define TC_DEBUG_COLLECT(s) \
    do {                    \
    } while (0)
#endif

// ---------------------------------------------------------------- helpers
// Edge flags, one bit per CSR position.  Bits only ever turn on, so a read
// that may be stale can only under-report set bits: an OR is issued only
// when the word read lacks one of the bits, which skips the many repeated
// settings of an edge that lies in several triangles.
// Sets bits of a flag word: one atomic OR whose result is not used, so the
// thread does not wait for it.  (Reading the word first to skip the atomic
// when its bits are already set made every count slower: the read is a
// dependent global load on the hot path.)
__device__ __forceinline__ void flag_or(uint32_t* __restrict__ fb, int64_t word, uint32_t mask) {
    atomicOr(&fb[word], mask);
}
__device__ __forceinline__ void flag_set(uint32_t* __restrict__ fb, int64_t p) {
    flag_or(fb, p >> 5, 1u << (p & 31));
}
__device__ __forceinline__ bool flag_get(const uint32_t* __restrict__ fb, int64_t p) {
    return (fb[p >> 5] >> (p & 31)) & 1u;
}
inline int64_t flag_words(int64_t e2) { return (e2 >> 5) + 4; }
inline tc_dims dims_of(const tc_graph* g) { return tc_dims{g->n, 2 * g->m, flag_words(2 * g->m)}; }

namespace tcx {

// Status of a CUDA runtime result.
tc_status from_cuda(cudaError_t e);

// Stream-ordered allocation from the device pool (no implicit sync).
tc_status dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

// Launch accounting and optional per-kernel event timing.
void add_launches(int64_t k);   // counts launches made without note_launch
// Kernels one call of a library routine (CUB) launches, for the launch
// count: the call is captured once per (site, size, bits) into a graph on a
// private stream — capturing records the launches without running them —
// and the graph's kernel nodes are counted.
int64_t library_kernels(const char* site, int64_t size, int64_t bits,
                        const std::function<cudaError_t(cudaStream_t)>& call);
// Runs a library call on s and adds its kernels to the launch count (less
// one when a launch_scope around it already counted the site).
template <class F>
tc_status run_library(const char* site, int64_t size, int64_t bits, bool in_scope, cudaStream_t s, F call) {
    const int64_t k = library_kernels(site, size, bits, std::function<cudaError_t(cudaStream_t)>(call));
    const cudaError_t e = call(s);
    if (e != cudaSuccess) return from_cuda(e);
    add_launches(in_scope ? k - 1 : k);
    return TC_OK;
}
// phase 0 before, 1 after; counts = false times a copy without counting a launch
void note_launch(const char* name, cudaStream_t s, int phase, bool counts = true);
// NVTX range over a host scope (entry points, library phases): shows on a
// profiler's timeline; without a profiler attached a push/pop costs a few ns.
struct nvtx_range {
    explicit nvtx_range(const char* name) { nvtxRangePushA(name); }
    ~nvtx_range() { nvtxRangePop(); }
};
struct launch_scope {
    const char* name; cudaStream_t s;
    launch_scope(const char* n, cudaStream_t st) : name(n), s(st) {
        nvtxRangePushA(name);
        note_launch(name, s, 0);
    }
    ~launch_scope() {
        note_launch(name, s, 1);
        nvtxRangePop();
    }
};
// Times the copies issued inside it under `name` (profile entries named
// "copy_*"); they are not kernel launches.
struct copy_scope {
    const char* name; cudaStream_t s;
    copy_scope(const char* n, cudaStream_t st) : name(n), s(st) { note_launch(name, s, 0, false); }
    ~copy_scope() { note_launch(name, s, 1, false); }
};

int sm_count();

// build pieces (tc_build.cu)
tc_status build_graph(tc_graph* g, const void* src, const void* dst, int64_t np, int64_t n,
                      uint32_t flags, cudaStream_t s);
void free_graph_memory(tc_graph* g);

// dense core (tc_core.cu).  Build flag for unions of many graphs, which
// have no dense core: the build never sets one up.
constexpr uint32_t TC_BUILD_NO_CORE = 1u << 30;
// Chooses the core (g->core_c) from d_H of the top ranks (dh, device),
// before the head records are written: those whose lower end is in the core
// get stream length 0.
tc_status core_setup(tc_graph* g, const int32_t* dh, uint32_t flags, cudaStream_t s);
// Adds the core's triangles: △ of its vertices, △(G), and flags (or, with
// edge counts, t(u, v)) of its edges.
tc_status run_core(tc_graph* g, cudaStream_t s, bool edge_counts);

// count (tc_count.cu)
tc_status make_plan(tc_graph* g, int strategy, cudaStream_t s);
void free_plan(tc_plan& p, cudaStream_t s);
// edge_counts: t(u, v) into g->ecnt; shard k of num_shards counts only the
// items k, k + num_shards, ... of every class (partial counts and flags)
tc_status run_count(tc_graph* g, cudaStream_t s, bool edge_counts = false, int shard = 0, int num_shards = 1);
// gather + divide (tc_gather.cu)
tc_status run_centrality(tc_graph* g, uint64_t* d_numer, double* d_tc, cudaStream_t s);
tc_status run_graph_sums(tc_graph* g, const int32_t* rank_graph, unsigned long long* sums, cudaStream_t s);
tc_status run_divide(const uint64_t* d_numer, int64_t n, uint64_t den, double* d_tc, cudaStream_t s);
tc_status export_tri(tc_graph* g, uint64_t* d_tri, cudaStream_t s);
tc_status export_flags(tc_graph* g, uint8_t* d_flag, cudaStream_t s);
tc_status export_edge_counts(tc_graph* g, uint32_t* d_out, cudaStream_t s);
// loads △(v) (caller labels) and canonical edge flags; counters[0] = Σ △(v)
tc_status import_counts(tc_graph* g, const uint64_t* d_tri, const uint8_t* d_flag, cudaStream_t s);

}  // namespace tcx

