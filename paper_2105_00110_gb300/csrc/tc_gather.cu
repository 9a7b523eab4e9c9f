// tc_centrality: the per-vertex gather and the one division of step 3 of
// the elementary algorithm (section "Algorithm"; Algorithm 2).
//
// Algorithm 2 forms x = Σ_{u∈N△[v]} △(u) (core sum, v included),
// s = Σ_{u∈N(v)} △(u) and y = s − x + △(v), then (x/3 + y)/△(G).  Here the
// same quantity is kept exact as one integer
//     numer(v) = x + 3y = △(v) + Σ_{u∈N(v)} (u ∈ N△(v) ? 1 : 3) · △(u)
// and divided once by 3△(G).  u ∈ N△(v) is the edge flag of (v, u): for a
// tail entry of row v (u above v) the flag sits at the entry itself, for a
// head entry (u below v) at its twin, the canonical entry in row u.
#include <algorithm>

#include "tc_internal.cuh"

namespace tcx {

namespace {

typedef unsigned long long ull;

// a / b correctly rounded (nearest, ties to even).  Operands below 2^53 are
// exact doubles, so one IEEE division is the answer.  Otherwise the
// quotient is developed in base-2^64 digits (integer part, then two
// fraction digits by 128-by-64-bit division), which always holds at least
// 54 significant bits because a/b >= 2^-64 when a >= 1; the bits below
// them and the last remainder form the sticky bit.
__device__ double div_rn(ull a, ull b) {
    if (b == 0) return __longlong_as_double(0x7ff8000000000000ll);
    if (a == 0) return 0.0;
    const ull lim = 1ull << 53;
    if (a < lim && b < lim) return __ddiv_rn((double)a, (double)b);
    ull q = a / b, r = a % b;
    unsigned __int128 t = (unsigned __int128)r << 64;
    ull f1 = (ull)(t / b);
    r = (ull)(t % b);
    t = (unsigned __int128)r << 64;
    ull f2 = (ull)(t / b);
    r = (ull)(t % b);
    bool sticky = r != 0;
    unsigned __int128 win;
    int k, lead;   // lead: position of the leading one counted from the fraction's start
    if (q) {
        k = 63 - __clzll((long long)q);
        win = ((unsigned __int128)q << 64) | f1;   // digits q.f1
        lead = 64 + k;
        sticky |= f2 != 0;
    } else {
        k = 63 - __clzll((long long)f1);
        win = ((unsigned __int128)f1 << 64) | f2;  // digits 0.f1 f2
        lead = 64 + k;
    }
    const int shift = lead - 53;                  // keep 54 bits: 53 + rounding bit
    ull m54 = (ull)(win >> shift);
    sticky |= (win & (((unsigned __int128)1 << shift) - 1)) != 0;
    // value of the lowest kept bit: q-case 2^(k-53); f-case 2^(k-53-64)
    int e = q ? (k - 53) : (k - 53 - 64);
    ull rb = m54 & 1;
    ull mant = m54 >> 1;
    e += 1;
    if (rb && (sticky || (mant & 1))) mant += 1;
    return ldexp((double)mant, e);
}

__device__ __forceinline__ ull warp_sum(ull x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// numer(r) = △(r) + Σ_{u ∈ N(r)} (u ∈ N△(r) ? 1 : 3)·△(u).  A tail entry
// holds u in col and its flag in place; a head entry's record holds u and
// the twin position where its flag sits.
// Rows are in rank (= degree) order, so three contiguous rank bands get
// one thread, one warp and one CTA per row.
struct gather_args;
__device__ __forceinline__ void finish_row(int64_t r, ull acc, const gather_args& a);

struct gather_args {
    const int64_t* row_ptr;
    const int64_t* hstart;
    const int32_t* col;
    const tc_head* head;
    const uint32_t* flag;
    const ull* tri;
    const int32_t* perm;
    ull den;
    const int32_t* rank_graph;   // batches: graph of each rank, or null
    const ull* den_graph;        // batches: 3△ of each graph
    const uint32_t* tri32;       // △ in 32 bits (half the size of tri: stays in L2), or the
                                 // escape 0xffffffff where △ >= 2^32
    ull* numer_out;
    double* tc_out;
    tc_dims dm;
};

// △(u) of a neighbour: the 32-bit copy, or the full count behind its escape.
__device__ __forceinline__ ull tri_of(const gather_args& a, int32_t u) {
    const uint32_t t = a.tri32[TC_IX(u, a.dm.n)];
    return t != 0xffffffffu ? (ull)t : a.tri[TC_IX(u, a.dm.n)];
}

// One adjacency entry's term (flag ? 1 : 3)·△(u): a head entry's record
// gives u and the twin position holding its flag, a tail entry holds u in
// col and its flag in place.
__device__ __forceinline__ ull head_term(const gather_args& a, int64_t p) {
    const tc_head rec = a.head[TC_IX(p, a.dm.e2)];
    return (flag_get(a.flag, TC_IX(rec.twin, a.dm.fw * 32)) ? 1ull : 3ull) * tri_of(a, rec.u);
}
__device__ __forceinline__ ull tail_term(const gather_args& a, int64_t p) {
    return (flag_get(a.flag, TC_IX(p, a.dm.fw * 32)) ? 1ull : 3ull) * tri_of(a, a.col[TC_IX(p, a.dm.e2)]);
}

__global__ void k_tri32(const ull* __restrict__ tri, int64_t n, uint32_t* __restrict__ tri32) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        tri32[r] = tri[r] < 0xffffffffull ? (uint32_t)tri[r] : 0xffffffffu;
}

__device__ __forceinline__ void finish_row(int64_t r, ull acc, const gather_args& a) {
    const int32_t v = a.perm[TC_IX(r, a.dm.n)];
    if (a.numer_out) a.numer_out[v] = acc;
    if (a.tc_out) a.tc_out[v] = div_rn(acc, a.rank_graph ? a.den_graph[a.rank_graph[r]] : a.den);
}

// one thread per row, rows [r0, r1)
__global__ void __launch_bounds__(256) k_gather_thread(gather_args a, int64_t r0, int64_t r1) {
    for (int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < r1;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = a.row_ptr[r], h = a.hstart[r], e = a.row_ptr[r + 1];
        ull acc = a.tri[r];
        for (int64_t p = b; p < h; ++p) acc += head_term(a, p);
        for (int64_t p = h; p < e; ++p) acc += tail_term(a, p);
        finish_row(r, acc, a);
    }
}

// one warp per row, rows [r0, r1)
__global__ void __launch_bounds__(256) k_gather_warp(gather_args a, int64_t r0, int64_t r1) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = r0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); r < r1; r += warps) {
        const int64_t b = a.row_ptr[r], h = a.hstart[r], e = a.row_ptr[r + 1];
        ull acc = 0;
        for (int64_t p = b + lane; p < h; p += 32) acc += head_term(a, p);
        for (int64_t p = h + lane; p < e; p += 32) acc += tail_term(a, p);
        acc = warp_sum(acc);
        if (lane == 0) finish_row(r, acc + a.tri[r], a);
    }
}

// one CTA per row, rows [r0, r1)
__global__ void __launch_bounds__(1024) k_gather_cta(gather_args a, int64_t r0, int64_t r1) {
    __shared__ ull part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r = r0 + blockIdx.x; r < r1; r += gridDim.x) {
        const int64_t b = a.row_ptr[r], h = a.hstart[r], e = a.row_ptr[r + 1];
        ull acc = 0;
        for (int64_t p = b + threadIdx.x; p < h; p += blockDim.x) acc += head_term(a, p);
        for (int64_t p = h + threadIdx.x; p < e; p += blockDim.x) acc += tail_term(a, p);
        acc = warp_sum(acc);
        if (lane == 0) part[warp] = acc;
        __syncthreads();
        if (warp == 0) {
            ull x = lane < (int)(blockDim.x >> 5) ? part[lane] : 0ull;
            x = warp_sum(x);
            if (lane == 0) finish_row(r, x + a.tri[r], a);
        }
        __syncthreads();
    }
}

// Σ_{v ∈ graph k} △(v) (= 3△(G_k)) for every graph of a batch; lanes of a
// warp that hit the same graph add once.
__global__ void k_graph_sums(const ull* __restrict__ tri, const int32_t* __restrict__ rank_graph, int64_t n,
                             ull* __restrict__ sums) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = rank_graph[r];
        const ull t = tri[r];
        const unsigned same = __match_any_sync(__activemask(), k);
        ull sum = 0;
        for (unsigned mm = same; mm; mm &= mm - 1) sum += __shfl_sync(same, t, __ffs(mm) - 1);
        if ((threadIdx.x & 31) == __ffs(same) - 1 && sum) atomicAdd(&sums[k], sum);
    }
}

__global__ void k_divide(const ull* __restrict__ numer, int64_t n, ull den, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = div_rn(numer[i], den);
}

__global__ void k_export_tri(const ull* __restrict__ tri, const int32_t* __restrict__ perm,
                             int64_t n, ull* __restrict__ out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        out[perm[r]] = tri[r];
}

__global__ void k_export_flags(const uint32_t* __restrict__ flag, const int64_t* __restrict__ edge_tail,
                               int64_t m, uint8_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = flag_get(flag, edge_tail[e]) ? 1 : 0;
}

__global__ void k_export_edge_counts(const uint32_t* __restrict__ ecnt, const int64_t* __restrict__ edge_tail,
                                     int64_t m, uint32_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = ecnt[edge_tail[e]];
}

// Counts and flags handed back in the public layout (caller labels,
// canonical edge order), e.g. summed / OR-ed over shards: △(v) into rank
// space with their sum, flags onto the tail entries.
__global__ void k_import_tri(const uint64_t* __restrict__ in, const int32_t* __restrict__ perm, int64_t n,
                             ull* __restrict__ tri, ull* __restrict__ sum) {
    ull local = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const ull x = in[perm[r]];
        tri[r] = x;
        local += x;
    }
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(sum, local);
}

__global__ void k_import_flags(const uint8_t* __restrict__ in, const int64_t* __restrict__ edge_tail, int64_t m,
                               uint32_t* __restrict__ flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        if (in[e]) flag_set(flag, edge_tail[e]);
}

inline int blocks_for(int64_t items, int threads) {
    int64_t b = (items + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * 16;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace

tc_status run_centrality(tc_graph* g, uint64_t* d_numer, double* d_tc, cudaStream_t s) {
    const int64_t n = g->n;
    if (n == 0) return TC_OK;
    gather_args a{g->row_ptr, g->hstart, g->col, g->head, g->flag, g->tri, g->perm,
                  3ull * (ull)g->total, g->rank_graph, g->den_graph, g->tri32, (ull*)d_numer, d_tc,
                  dims_of(g)};
    {
        launch_scope ls("gather_tri32", s);
        k_tri32<<<blocks_for(n, 256), 256, 0, s>>>(g->tri, n, g->tri32);
        TC_LAUNCH_CHECK();
    }
    const int64_t r1 = g->band[0], r2 = g->band[1];   // degree <= 32 | <= 4096 | larger
    if (r1 > 0) {
        launch_scope ls("gather_thread", s);
        k_gather_thread<<<blocks_for(r1, 256), 256, 0, s>>>(a, 0, r1);
        TC_LAUNCH_CHECK();
    }
    if (r2 > r1) {
        launch_scope ls("gather_warp", s);
        k_gather_warp<<<blocks_for((r2 - r1) * 32, 256), 256, 0, s>>>(a, r1, r2);
        TC_LAUNCH_CHECK();
    }
    if (n > r2) {
        launch_scope ls("gather_cta", s);
        const int64_t rows = n - r2;
        k_gather_cta<<<(int)std::min<int64_t>(rows, (int64_t)sm_count() * 2), 1024, 0, s>>>(a, r2, n);
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}

tc_status run_graph_sums(tc_graph* g, const int32_t* rank_graph, ull* sums, cudaStream_t s) {
    if (g->n == 0) return TC_OK;
    launch_scope ls("batch_graph_sums", s);
    k_graph_sums<<<blocks_for(g->n, 256), 256, 0, s>>>(g->tri, rank_graph, g->n, sums);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status run_divide(const uint64_t* d_numer, int64_t n, uint64_t den, double* d_tc, cudaStream_t s) {
    if (n == 0) return TC_OK;
    launch_scope ls("divide", s);
    k_divide<<<blocks_for(n, 256), 256, 0, s>>>((const ull*)d_numer, n, (ull)den, d_tc);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status export_tri(tc_graph* g, uint64_t* d_tri, cudaStream_t s) {
    if (g->n == 0) return TC_OK;
    launch_scope ls("export_tri", s);
    k_export_tri<<<blocks_for(g->n, 256), 256, 0, s>>>(g->tri, g->perm, g->n, (ull*)d_tri);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status export_edge_counts(tc_graph* g, uint32_t* d_out, cudaStream_t s) {
    if (g->m == 0) return TC_OK;
    if (!g->ecnt) return TC_ERR_STATE;
    launch_scope ls("export_edge_counts", s);
    k_export_edge_counts<<<blocks_for(g->m, 256), 256, 0, s>>>(g->ecnt, g->edge_tail, g->m, d_out);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status import_counts(tc_graph* g, const uint64_t* d_tri, const uint8_t* d_flag, cudaStream_t s) {
    const int64_t n = g->n, m = g->m;
    TC_CUDA(cudaMemsetAsync(g->counters, 0, 8 * 8, s));
    TC_CUDA(cudaMemsetAsync(g->flag, 0, flag_words(2 * m) * 4, s));
    if (n > 0) {
        launch_scope ls("import_tri", s);
        k_import_tri<<<blocks_for(n, 256), 256, 0, s>>>(d_tri, g->perm, n, g->tri, g->counters);
        TC_LAUNCH_CHECK();
    }
    if (m > 0) {
        launch_scope ls("import_flags", s);
        k_import_flags<<<blocks_for(m, 256), 256, 0, s>>>(d_flag, g->edge_tail, m, g->flag);
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}

tc_status export_flags(tc_graph* g, uint8_t* d_flag, cudaStream_t s) {
    if (g->m == 0) return TC_OK;
    launch_scope ls("export_flags", s);
    k_export_flags<<<blocks_for(g->m, 256), 256, 0, s>>>(g->flag, g->edge_tail, g->m, d_flag);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace tcx
