// tc_build_csr: simple undirected graph, degree order π, orientation and
// the count-step plan, all on the device.
//
//  1. pairs -> canonical keys (min, max); self-loops become a sentinel
//     (the set-up of section "Comparison": symmetrised, loop-free, simple)
//  2. radix sort + unique -> the m undirected edges, caller labels
//  3. degrees; π = sort by (degree, label) (section "Notation")
//  4. both directions of every edge relabelled by π, radix sorted ->
//     symmetric CSR in rank space, rows ascending, so each row is
//     [N_L(v) | N_H(v)] (Lemma 1's partition, done by sorting)
//  5. hstart (row split), edge_tail, twin and hrem of every head entry
//  6. planner: per middle vertex v its work W(v) = Σ_{u∈N_L(v)} hrem, and
//     the work items of the count step, heavy vertices split into chunks
//
// Radix sorts and scans use CUB (header-only, compiled into this library).
#include <cub/cub.cuh>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tc_internal.cuh"

namespace tcx {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int per_thread = 1) {
    int64_t want = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
    int64_t cap = (int64_t)sm_count() * 16;
    if (want < 1) want = 1;
    return (int)std::min(want, cap);
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

template <typename T>
__global__ void k_make_keys(const T* __restrict__ src, const T* __restrict__ dst, int64_t np,
                            int64_t n, int bits, uint64_t* __restrict__ keys,
                            unsigned int* __restrict__ err) {
    GRID_STRIDE(i, np) {
        int64_t a = (int64_t)src[i], b = (int64_t)dst[i];
        uint64_t key = ~0ull;
        if (a < 0 || b < 0 || a >= n || b >= n) {
            atomicOr(err, 1u);
        } else if (a != b) {
            uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
            key = (lo << bits) | hi;
        }
        keys[i] = key;
    }
}

__global__ void k_edges_degrees(const uint64_t* __restrict__ ukeys, int64_t m, int bits,
                                int32_t* __restrict__ eu, int32_t* __restrict__ ev,
                                int32_t* __restrict__ deg) {
    const uint64_t mask = (1ull << bits) - 1;
    GRID_STRIDE(e, m) {
        uint64_t k = ukeys[e];
        int32_t u = (int32_t)(k >> bits), v = (int32_t)(k & mask);
        eu[e] = u;
        ev[e] = v;
        // edges are sorted by u: lanes with the same u add their count once
        const unsigned same = __match_any_sync(__activemask(), u);
        if ((threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&deg[u], __popc(same));
        atomicAdd(&deg[v], 1);
    }
}

__global__ void k_rank_keys(const int32_t* __restrict__ deg, int64_t n, int bits,
                            uint64_t* __restrict__ keys) {
    GRID_STRIDE(v, n) keys[v] = ((uint64_t)deg[v] << bits) | (uint64_t)v;
}

__global__ void k_rank_apply(const uint64_t* __restrict__ sorted, int64_t n, int bits,
                             int32_t* __restrict__ perm, int32_t* __restrict__ rank,
                             int64_t* __restrict__ degr) {
    const uint64_t mask = (1ull << bits) - 1;
    GRID_STRIDE(r, n) {
        uint64_t k = sorted[r];
        int32_t v = (int32_t)(k & mask);
        perm[r] = v;
        rank[v] = (int32_t)r;
        degr[r] = (int64_t)(k >> bits);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) degr[n] = 0;
}

// Every undirected edge once in rank space: key (lo, hi) with lo < hi the
// ranks of its ends, value its canonical id; d_H(lo) counted.
__global__ void k_edge_rank_keys(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                 const int32_t* __restrict__ rank, int64_t m, int bits,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                 int32_t* __restrict__ dh) {
    GRID_STRIDE(e, m) {
        const uint64_t ru = (uint64_t)rank[eu[e]], rv = (uint64_t)rank[ev[e]];
        const uint64_t lo = ru < rv ? ru : rv, hi = ru < rv ? rv : ru;
        keys[e] = (lo << bits) | hi;
        vals[e] = (uint32_t)e;
        atomicAdd(&dh[lo], 1);
    }
}

// Row split: the last d_H(r) entries of row r hold N_H(r).
__global__ void k_hstart(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ dh, int64_t n,
                         int64_t* __restrict__ hstart) {
    GRID_STRIDE(r, n) hstart[r] = row_ptr[r + 1] - dh[r];
}

// Writes both entries of every edge.  The edges arrive sorted by (lo, hi),
// so the tail entry (row lo, N_H(lo) ascending) of the i-th edge is at
// hstart[lo] + (i - hptr[lo]); the head entry (row hi, N_L(hi) in any
// order) takes the next free slot of row hi's head as the record
// {lo, |{w ∈ N_H(lo) : w > hi}|, tail position}.
__global__ void k_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t m,
                          int bits, const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                          const int64_t* __restrict__ hptr, int32_t* __restrict__ hcur,
                          int32_t* __restrict__ col, tc_head* __restrict__ head,
                          int64_t* __restrict__ edge_tail) {
    const uint64_t mask = (1ull << bits) - 1;
    GRID_STRIDE(i, m) {
        const uint64_t k = keys[i];
        const int64_t lo = (int64_t)(k >> bits), hi = (int64_t)(k & mask);
        const int64_t tail = hstart[lo] + (i - hptr[lo]);
        col[tail] = (int32_t)hi;
        edge_tail[vals[i]] = tail;
        const int64_t hp = row_ptr[hi] + atomicAdd(&hcur[hi], 1);
        tc_head rec;
        rec.u = (int32_t)lo;
        rec.hrem = (int32_t)(row_ptr[lo + 1] - tail - 1);
        rec.twin = tail;
        head[hp] = rec;   // one 16-byte store
    }
}

// First ranks whose degree exceeds 32 and 4096 (degrees ascend with rank).
__global__ void k_bands(const int64_t* __restrict__ row_ptr, int64_t n, int64_t* __restrict__ band) {
    const int64_t lim[2] = {32, 4096};
    for (int k = 0; k < 2; ++k) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (row_ptr[mid + 1] - row_ptr[mid] > lim[k]) hi = mid; else lo = mid + 1;
        }
        band[k] = lo;
    }
}

// ------------------------------------------------------------ row work
struct row_stats {
    unsigned long long sum_h2, wedges, sum_dh, max_h, max_d;
};

// One warp per row: W(v) = Σ_{u ∈ N_L(v)} hrem(u, v), the number of ids the
// count step streams for middle vertex v; plus shape statistics.
__global__ void k_row_work(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                           const tc_head* __restrict__ head, int64_t n, int64_t* __restrict__ work,
                           row_stats* __restrict__ st) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long l_h2 = 0, l_w = 0, l_dh = 0, l_maxh = 0, l_maxd = 0;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int64_t b = row_ptr[r], h = hstart[r], e = row_ptr[r + 1];
        unsigned long long w = 0;
        for (int64_t p = b + lane; p < h; p += 32) w += (unsigned long long)head[p].hrem;
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) {
            const unsigned long long hv = (unsigned long long)(e - h), d = (unsigned long long)(e - b);
            work[r] = (int64_t)w;
            l_h2 += hv * hv;
            l_w += w;
            l_dh += d * hv;
            l_maxh = l_maxh > hv ? l_maxh : hv;
            l_maxd = l_maxd > d ? l_maxd : d;
        }
    }
    if (lane == 0) {
        atomicAdd(&st->sum_h2, l_h2);
        atomicAdd(&st->wedges, l_w);
        atomicAdd(&st->sum_dh, l_dh);
        atomicMax(&st->max_h, l_maxh);
        atomicMax(&st->max_d, l_maxd);
    }
}

int bits_for(int64_t n) {
    int b = 1;
    while (b < 62 && ((int64_t)1 << b) < n) ++b;
    return b;
}

// Owns every temporary of a build so that an early return releases them.
struct scratch {
    cudaStream_t s;
    std::vector<void*> p;
    explicit scratch(cudaStream_t st) : s(st) { p.reserve(64); }
    template <typename T>
    tc_status get(T** out, size_t count) {
        void* q = nullptr;
        *out = nullptr;
        TC_TRY(dalloc(&q, count * sizeof(T) + 16, s));
        p.push_back(q);
        *out = (T*)q;
        return TC_OK;
    }
    ~scratch() {
        for (void* q : p) dfree(q, s);
    }
};

template <typename T>
tc_status sort_keys(scratch& sc, cub::DoubleBuffer<T>& buf, int64_t count, int end_bit, cudaStream_t s) {
    size_t bytes = 0;
    TC_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, bytes, buf, count, 0, end_bit, s));
    uint8_t* tmp = nullptr;
    TC_TRY(sc.get(&tmp, bytes));
    TC_CUDA(cub::DeviceRadixSort::SortKeys(tmp, bytes, buf, count, 0, end_bit, s));
    return TC_OK;
}

}  // namespace

void free_graph_memory(tc_graph* g) {
    cudaStream_t s = g->stream;
    void* ptrs[] = {g->edge_u, g->edge_v, g->perm, g->row_ptr, g->col, g->hstart, g->head,
                    g->edge_tail, g->work, g->tri, g->flag, g->numer, g->counters};
    for (void* q : ptrs) dfree(q, s);
    free_plan(g->plan, s);
}

tc_status build_graph(tc_graph* g, const void* src, const void* dst, int64_t np, int64_t n,
                      uint32_t flags, cudaStream_t s) {
    g->n = n;
    g->bits = bits_for(n);
    g->stream = s;
    const int bits = g->bits;
    const bool i32 = (flags & TC_IDS_INT32) != 0;
    const size_t id_bytes = i32 ? 4 : 8;
    scratch sc(s);

    // ---- 0. inputs on the device
    const void* dsrc = src;
    const void* ddst = dst;
    if (!(flags & TC_IN_DEVICE) && np > 0) {
        void *a = nullptr, *b = nullptr;
        TC_TRY(sc.get((uint8_t**)&a, np * id_bytes));
        TC_TRY(sc.get((uint8_t**)&b, np * id_bytes));
        TC_CUDA(cudaMemcpyAsync(a, src, np * id_bytes, cudaMemcpyHostToDevice, s));
        TC_CUDA(cudaMemcpyAsync(b, dst, np * id_bytes, cudaMemcpyHostToDevice, s));
        dsrc = a;
        ddst = b;
    }

    // ---- 1-2. canonical undirected edges
    unsigned int* err = nullptr;
    TC_TRY(sc.get(&err, 4));
    TC_CUDA(cudaMemsetAsync(err, 0, 4, s));
    uint64_t *ka = nullptr, *kb = nullptr;
    int64_t m = 0;
    int64_t* d_nsel = nullptr;
    TC_TRY(sc.get(&d_nsel, 2));
    if (np > 0) {
        TC_TRY(sc.get(&ka, np));
        TC_TRY(sc.get(&kb, np));
        {
            launch_scope ls("build_make_keys", s);
            if (i32)
                k_make_keys<int32_t><<<grid_for(np), kThreads, 0, s>>>(
                    (const int32_t*)dsrc, (const int32_t*)ddst, np, n, bits, ka, err);
            else
                k_make_keys<int64_t><<<grid_for(np), kThreads, 0, s>>>(
                    (const int64_t*)dsrc, (const int64_t*)ddst, np, n, bits, ka, err);
            TC_LAUNCH_CHECK();
        }
        cub::DoubleBuffer<uint64_t> kbuf(ka, kb);
        {
            launch_scope ls("build_sort_pairs", s);
            TC_TRY(sort_keys(sc, kbuf, np, 2 * bits, s));
        }
        uint64_t* sorted = kbuf.Current();
        uint64_t* uniq = kbuf.Alternate();
        size_t bytes = 0;
        TC_CUDA(cub::DeviceSelect::Unique(nullptr, bytes, sorted, uniq, d_nsel, np, s));
        uint8_t* tmp = nullptr;
        TC_TRY(sc.get(&tmp, bytes));
        {
            launch_scope ls("build_unique", s);
            TC_CUDA(cub::DeviceSelect::Unique(tmp, bytes, sorted, uniq, d_nsel, np, s));
        }
        int64_t h_sel = 0;
        uint64_t last = 0;
        unsigned int h_err = 0;
        TC_CUDA(cudaMemcpyAsync(&h_sel, d_nsel, 8, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        if (h_err) return TC_ERR_INVALID_ARG;
        if (h_sel > 0) {
            TC_CUDA(cudaMemcpyAsync(&last, uniq + h_sel - 1, 8, cudaMemcpyDeviceToHost, s));
            TC_CUDA(cudaStreamSynchronize(s));
        }
        m = h_sel - ((h_sel > 0 && last == ~0ull) ? 1 : 0);
        ka = uniq;  // the m unique keys
    }
    if (m >= ((int64_t)1 << 32)) return TC_ERR_INVALID_ARG;  // edge ids are 32-bit
    g->m = m;
    const int64_t e2 = 2 * m;

    // ---- graph-owned arrays
    TC_TRY(dalloc((void**)&g->edge_u, (m + 1) * 4, s));
    TC_TRY(dalloc((void**)&g->edge_v, (m + 1) * 4, s));
    TC_TRY(dalloc((void**)&g->perm, (n + 1) * 4, s));
    TC_TRY(dalloc((void**)&g->row_ptr, (n + 2) * 8, s));
    // 32 ids of padding: the count step reads whole groups of 16-byte
    // units, and the last group of the last row may extend past 2m
    TC_TRY(dalloc((void**)&g->col, (e2 + 32) * 4, s));
    TC_CUDA(cudaMemsetAsync(g->col + e2, 0xff, 32 * 4, s));
    TC_TRY(dalloc((void**)&g->hstart, (n + 1) * 8, s));
    TC_TRY(dalloc((void**)&g->head, (e2 + 1) * sizeof(tc_head), s));
    TC_TRY(dalloc((void**)&g->edge_tail, (m + 1) * 8, s));
    TC_TRY(dalloc((void**)&g->tri, (n + 1) * 8, s));
    TC_TRY(dalloc((void**)&g->numer, (n + 1) * 8, s));
    TC_TRY(dalloc((void**)&g->flag, flag_words(e2) * 4, s));
    TC_TRY(dalloc((void**)&g->counters, 8 * 8, s));

    // ---- 3. degrees and the order π
    int32_t* deg = nullptr;
    TC_TRY(sc.get(&deg, n + 1));
    TC_CUDA(cudaMemsetAsync(deg, 0, (n + 1) * 4, s));
    if (m > 0) {
        launch_scope ls("build_edges_degrees", s);
        k_edges_degrees<<<grid_for(m), kThreads, 0, s>>>(ka, m, bits, g->edge_u, g->edge_v, deg);
        TC_LAUNCH_CHECK();
    }
    int32_t* rank = nullptr;
    int64_t* degr = nullptr;
    TC_TRY(sc.get(&rank, n + 1));
    TC_TRY(sc.get(&degr, n + 2));
    if (n > 0) {
        uint64_t *ra = nullptr, *rb = nullptr;
        TC_TRY(sc.get(&ra, n));
        TC_TRY(sc.get(&rb, n));
        {
            launch_scope ls("build_rank_keys", s);
            k_rank_keys<<<grid_for(n), kThreads, 0, s>>>(deg, n, bits, ra);
            TC_LAUNCH_CHECK();
        }
        cub::DoubleBuffer<uint64_t> rbuf(ra, rb);
        {
            launch_scope ls("build_sort_rank", s);
            TC_TRY(sort_keys(sc, rbuf, n, 2 * bits, s));
        }
        launch_scope ls("build_rank_apply", s);
        k_rank_apply<<<grid_for(n), kThreads, 0, s>>>(rbuf.Current(), n, bits, g->perm, rank, degr);
        TC_LAUNCH_CHECK();
    } else {
        TC_CUDA(cudaMemsetAsync(degr, 0, 8, s));
    }
    {
        size_t bytes = 0;
        TC_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, degr, g->row_ptr, n + 1, s));
        uint8_t* tmp = nullptr;
        TC_TRY(sc.get(&tmp, bytes));
        launch_scope ls("build_row_ptr", s);
        TC_CUDA(cub::DeviceScan::ExclusiveSum(tmp, bytes, degr, g->row_ptr, n + 1, s));
    }

    // ---- 4. rank-space CSR: the m edges sorted once by (lo, hi) give every
    // N_H(r) in order; the heads N_L(r) need no order
    if (m > 0) {
        uint64_t *ka2 = nullptr, *kb2p = nullptr;
        uint32_t *va = nullptr, *vb = nullptr;
        int32_t *dh = nullptr, *hcur = nullptr;
        int64_t* hptr = nullptr;
        TC_TRY(sc.get(&ka2, m));
        TC_TRY(sc.get(&kb2p, m));
        TC_TRY(sc.get(&va, m));
        TC_TRY(sc.get(&vb, m));
        TC_TRY(sc.get(&dh, n + 1));
        TC_TRY(sc.get(&hcur, n + 1));
        TC_TRY(sc.get(&hptr, n + 1));
        TC_CUDA(cudaMemsetAsync(dh, 0, (n + 1) * 4, s));
        TC_CUDA(cudaMemsetAsync(hcur, 0, (n + 1) * 4, s));
        {
            launch_scope ls("build_edge_rank_keys", s);
            k_edge_rank_keys<<<grid_for(m), kThreads, 0, s>>>(g->edge_u, g->edge_v, rank, m, bits, ka2, va, dh);
            TC_LAUNCH_CHECK();
        }
        cub::DoubleBuffer<uint64_t> kb2(ka2, kb2p);
        cub::DoubleBuffer<uint32_t> vb2(va, vb);
        size_t bytes = 0;
        TC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb2, vb2, m, 0, 2 * bits, s));
        size_t sbytes = 0;
        TC_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, sbytes, dh, hptr, n + 1, s));
        uint8_t* tmp = nullptr;
        TC_TRY(sc.get(&tmp, std::max(bytes, sbytes)));
        {
            launch_scope ls("build_sort_edges", s);
            TC_CUDA(cub::DeviceRadixSort::SortPairs(tmp, bytes, kb2, vb2, m, 0, 2 * bits, s));
        }
        {
            launch_scope ls("build_hptr", s);
            TC_CUDA(cub::DeviceScan::ExclusiveSum(tmp, sbytes, dh, hptr, n + 1, s));
        }
        {
            launch_scope ls("build_hstart", s);
            k_hstart<<<grid_for(n), kThreads, 0, s>>>(g->row_ptr, dh, n, g->hstart);
            TC_LAUNCH_CHECK();
        }
        {
            launch_scope ls("build_scatter", s);
            k_scatter<<<grid_for(m), kThreads, 0, s>>>(kb2.Current(), vb2.Current(), m, bits, g->row_ptr,
                                                        g->hstart, hptr, hcur, g->col, g->head,
                                                        g->edge_tail);
            TC_LAUNCH_CHECK();
        }
    } else if (n > 0) {
        // no edges: every row is empty
        TC_CUDA(cudaMemsetAsync(g->hstart, 0, n * 8, s));
    }

    // ---- 6. per-row work, statistics and the count-step plan
    TC_TRY(dalloc((void**)&g->work, (n + 1) * 8, s));
    row_stats* dst_stats = nullptr;
    TC_TRY(sc.get(&dst_stats, 1));
    TC_CUDA(cudaMemsetAsync(dst_stats, 0, sizeof(row_stats), s));
    if (n > 0) {
        launch_scope ls("build_row_work", s);
        int blocks = (int)std::min<int64_t>((n * 32 + kThreads - 1) / kThreads, (int64_t)sm_count() * 16);
        k_row_work<<<std::max(blocks, 1), kThreads, 0, s>>>(g->row_ptr, g->hstart, g->head, n, g->work,
                                                            dst_stats);
        TC_LAUNCH_CHECK();
    }
    int64_t* d_band = nullptr;
    TC_TRY(sc.get(&d_band, 2));
    {
        launch_scope ls("build_bands", s);
        k_bands<<<1, 1, 0, s>>>(g->row_ptr, n, d_band);
        TC_LAUNCH_CHECK();
    }
    row_stats hst{};
    TC_CUDA(cudaMemcpyAsync(&hst, dst_stats, sizeof(row_stats), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaMemcpyAsync(g->band, d_band, sizeof(g->band), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    tc_graph_stats& S = g->stats;
    S.n = n;
    S.m = m;
    S.max_degree = (int64_t)hst.max_d;
    S.max_out_degree = (int64_t)hst.max_h;
    S.sum_out_degree_sq = (double)hst.sum_h2;
    S.wedges = (double)hst.wedges;
    S.avg_degeneracy = m ? (double)hst.sum_dh / (double)m : 0.0;
    // the count kernels keep stream lengths and staged indices in 16 bits;
    // |N_H(v)| <= sqrt(2m) makes this reachable only with m >= 2^31 edges
    if (S.max_out_degree >= 65536) return TC_ERR_INVALID_ARG;
    // Count step: stage N_H(v) once per middle vertex (4m), read each head
    // entry's label, twin and stream length (16m), stream every wedge id
    // (4 W), write the vertex counts (8n) and one flag byte per tail entry (m).
    S.count_bytes = 4.0 * m + 16.0 * m + 4.0 * S.wedges + 8.0 * n + 1.0 * m;
    // Gather: per vertex row_ptr, hstart, perm, △(v), numerator and TC out
    // (8+8+4+8+8+8); per adjacency entry its label and the neighbour's count
    // (4+8); per head entry twin and the mirrored flag (8+1); per tail entry
    // its flag (1).
    S.centrality_bytes = 44.0 * n + 12.0 * (double)e2 + 9.0 * m + 1.0 * m;
    TC_TRY(make_plan(g, g->strategy, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

}  // namespace tcx
