// Dense core of the count step.
//
// In degree order the highest ranks hold the hubs, and among the top C of
// them the adjacency is dense (R-MAT scale 24: density 0.13 at C = 16384).
// A triangle u < v < w whose lowest vertex u is in that core has all three
// vertices there.  The sparse count kernels skip exactly these triangles
// (their head entries (u, v) with u in the core stream nothing) and this
// file counts them edge by edge: on a core edge (x, y) the core triangles
// through it number
//
//   T(x, y) = |N_c(x) ∩ N_c(y)| = (A_c² ∘ A_c)(x, y),
//
// the matrix form T = A² ∘ A of section "Notation" restricted to the core
// adjacency A_c, evaluated only where A_c has an edge.  With every core row
// packed one bit per core vertex, that intersection is a word-wise AND and
// a population count over ⌈C/32⌉ words — the bitmap membership test of the
// sparse kernels applied to a whole row at once.  Then for every core edge
// with T > 0: △(x) and △(y) gain T/2 each once summed (a core triangle lies
// on two core edges at each of its vertices), △(G) gains ΣT / 3, and the
// edge is flagged (or t(x, y) gains T in edge-count mode).
//
// Layout (core-local index i = rank - (n - C)):
//   R[i][W]  uint32  row i of A_c, bit j of word w = edge (i, 32w + j);
//                    W = ⌈C/32⌉ rounded up to 128·{1, 2, 4, 8} (zero padded)
//   P[i][W]  uint16  members of N_H(i) (bits above i) in words < w, so that
//                    the tail position of an edge (i, y), y > i, is
//                    hstart + P[i][y/32] + the bits of word y/32 in (i, y)
//
// k_core_pairs stages a block of UB consecutive rows (the lower ends u) in
// shared memory and walks a range of upper ends v: word u0/32 of row v
// tells which u of the block are neighbours below v (A_c is symmetric), and
// for each such u one warp ANDs the two rows — row v held in registers,
// 16-byte loads — and reduces the population counts.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "tc_internal.cuh"

namespace tcx {

// -1: choose C from the graph (default), 0: never, > 0: the top C ranks.
std::atomic<long long> g_core_mode{-1};

namespace {

typedef unsigned long long ull;

constexpr int kCoreSizes[] = {4096, 8192, 16384, 32768};
constexpr int64_t kCoreMax = 32768;
constexpr int kPairThreads = 512;
constexpr int kPairWarps = kPairThreads / 32;
constexpr int kVChunk = 512;   // upper ends per work item
constexpr int kFillThreads = 256;

// Rough rates, used only to decide whether a core pays: ids streamed per
// ms by the bitmap count kernel (R-MAT scale 24: the 1.0e10 ids of the top
// 16384 ranks took 10 ms), and row words ANDed per ms by k_core_pairs
// (R-MAT scales 22 and 24: 2.8e9 - 4.3e9).
constexpr double kStreamIdsPerMs = 1.0e9;
constexpr double kWordsPerMs = 3.5e9;
constexpr double kFixedMs = 0.1;       // fill, staging, launches
constexpr double kMinGainMs = 0.5;

inline int64_t core_words(int64_t C) {
    int64_t w = 128;
    while (w * 32 < C) w <<= 1;
    return w;   // 128, 256, 512 or 1024 for C <= 32768
}
inline int core_ub(int64_t W) { return W <= 512 ? 32 : 16; }
inline size_t pair_smem(int64_t W) {
    const int ub = core_ub(W);
    return (size_t)ub * W * 4 + (size_t)ub * W * 2 + (size_t)ub * 8 + (size_t)ub * 4;
}

// One warp per core row i (rank r = t + i): its higher neighbours N_H(r)
// — all in the core, ascending at the tail positions of row r — set bit
// (i, j) and the mirror bit (j, i) of R (zeroed beforehand), so R gets
// every core edge both ways without reading the head part of any row.  The
// row's own bits, gathered in a per-warp buffer first, also give P.
__global__ void __launch_bounds__(kFillThreads)
k_core_fill(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart, const int32_t* __restrict__ col,
            int64_t t, int64_t C, int64_t W, uint32_t* __restrict__ R, uint16_t* __restrict__ P, tc_dims dm) {
    extern __shared__ __align__(16) uint32_t fill_buf[];
    const int lane = threadIdx.x & 31;
    uint32_t* buf = fill_buf + (threadIdx.x >> 5) * W;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int K = (int)(W >> 5);   // words per lane for the prefix counts
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < C; i += warps) {
        const int64_t r = t + i;
        const int64_t h = hstart[TC_IX(r, dm.n)], e = row_ptr[TC_IX(r, dm.n) + 1];
        for (int w = lane; w < W; w += 32) buf[w] = 0;
        __syncwarp();
        const uint32_t ibit = 1u << (i & 31);
        for (int64_t p = h + lane; p < e; p += 32) {
            const int64_t j = (int64_t)col[TC_IX(p, dm.e2)] - t;   // j > i
            atomicOr(&buf[TC_IX(j >> 5, W)], 1u << (j & 31));
            atomicOr(&R[TC_IX(j * W + (i >> 5), C * W)], ibit);
        }
        __syncwarp();
        for (int w = lane; w < W; w += 32)
            if (buf[w]) atomicOr(&R[i * W + w], buf[w]);
        // P: members of N_H(r) (every bit of buf lies above i) in the words
        // before each word
        uint32_t mine = 0;
        for (int k = 0; k < K; ++k) mine += __popc(buf[lane * K + k]);
        uint32_t incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += x;
        }
        uint32_t run = incl - mine;
        uint16_t* Pr = P + i * W;
        for (int k = 0; k < K; ++k) {
            const int w = lane * K + k;
            Pr[w] = (uint16_t)run;
            run += __popc(buf[w]);
        }
        __syncwarp();
    }
}

// Σ popc(ru[w] & rv[w]) over this lane's 4·KW words.  With TC_CORE_CSA the
// words are taken in threes through a carry-save adder — s = a ^ b ^ c and
// c' = majority(a, b, c) hold the same ones as a, b, c with c' counted twice
// — so 3 words cost 2 population counts (the carry-save step of Harley and
// Seal's population count); the leftover words are counted directly.
#ifndef TC_CORE_CSA
#define TC_CORE_CSA 1
#endif
template <int KW>
__device__ __forceinline__ uint32_t and_popc(const uint4* ru, const uint4* rv, int lane) {
    uint32_t ones = 0, twos = 0;
    uint32_t p0 = 0, p1 = 0;   // words waiting for a third
    int np = 0;                 // resolved at compile time (loops fully unrolled)
    auto take = [&](uint32_t c) {
        if (!TC_CORE_CSA) {
            ones += __popc(c);
        } else if (np == 2) {
            ones += __popc(p0 ^ p1 ^ c);
            twos += __popc((p0 & p1) | (c & (p0 ^ p1)));
            np = 0;
        } else if (np == 1) {
            p1 = c;
            np = 2;
        } else {
            p0 = c;
            np = 1;
        }
    };
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        const uint4 x = ru[lane + 32 * k];
        take(x.x & rv[k].x);
        take(x.y & rv[k].y);
        take(x.z & rv[k].z);
        take(x.w & rv[k].w);
    }
    if (np >= 1) ones += __popc(p0);
    if (np == 2) ones += __popc(p1);
    return ones + 2 * twos;
}

// Work item q: block a = q / nvch of UB lower ends u ∈ [u0, u0 + UB) and the
// chunk j = q % nvch of upper ends v ∈ [j·kVChunk, (j+1)·kVChunk) ∩ (u0, C).
template <int KW>
__global__ void __launch_bounds__(kPairThreads, 2)
k_core_pairs(const uint32_t* __restrict__ R, const uint16_t* __restrict__ P, const int64_t* __restrict__ hstart,
             int64_t t, int64_t C, int64_t nvch, int64_t nitems, ull* __restrict__ cursor,
             ull* __restrict__ S, uint32_t* __restrict__ flag, uint32_t* __restrict__ ecnt,
             ull* __restrict__ sum_t, tc_dims dm) {
    constexpr int W = 128 * KW;
    constexpr int UB = W <= 512 ? 32 : 16;
    extern __shared__ __align__(16) uint8_t pair_dyn[];
    uint32_t* Rs = (uint32_t*)pair_dyn;                  // [UB][W]
    uint16_t* Ps = (uint16_t*)(Rs + UB * W);             // [UB][W]
    int64_t* Hs = (int64_t*)(Ps + UB * W);               // [UB] hstart of the block's rows
    uint32_t* Su = (uint32_t*)(Hs + UB);                 // [UB] Σ T at each lower end, this item
    __shared__ int64_t s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ull all = 0;
    for (;;) {
        __syncthreads();   // the previous item's reads of the staged rows are done
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(cursor, 1ull);
        __syncthreads();
        const int64_t q = s_item;
        if (q >= nitems) break;
        const int64_t a = q / nvch, j = q % nvch;
        const int64_t u0 = a * UB;
        const int64_t vlo = j * kVChunk > u0 + 1 ? j * kVChunk : u0 + 1;
        const int64_t vhi = (j + 1) * kVChunk < C ? (j + 1) * kVChunk : C;
        if (vlo >= vhi) continue;
        const int nrows = (int)(C - u0 < UB ? C - u0 : UB);
        {
            const uint4* src = (const uint4*)(R + u0 * W);
            uint4* dst = (uint4*)Rs;
            for (int k = threadIdx.x; k < UB * W / 4; k += kPairThreads)
                dst[k] = k < nrows * W / 4 ? src[k] : make_uint4(0, 0, 0, 0);
            const uint4* psrc = (const uint4*)(P + u0 * W);
            uint4* pdst = (uint4*)Ps;
            for (int k = threadIdx.x; k < UB * W / 8; k += kPairThreads)
                pdst[k] = k < nrows * W / 8 ? psrc[k] : make_uint4(0, 0, 0, 0);
            if (threadIdx.x < UB) {
                Hs[threadIdx.x] = threadIdx.x < nrows ? hstart[TC_IX(t + u0 + threadIdx.x, dm.n)] : 0;
                Su[threadIdx.x] = 0;
            }
        }
        __syncthreads();
        const int uw = (int)(u0 >> 5), ush = (int)(u0 & 31);
        // the next upper end's mask word and row are loaded while this one
        // is processed (double-buffered in registers for rows of <= 512 words)
        constexpr bool kAhead = KW <= 4;
        uint32_t mask_n = 0;
        uint4 rv_n[KW];
        int64_t v = vlo + warp;
        auto fetch = [&](int64_t x, uint32_t& mk, uint4* rr) {
            const uint32_t* Rx = R + x * W;
            mk = __ldg(Rx + uw);
#pragma unroll
            for (int k = 0; k < KW; ++k) rr[k] = __ldg((const uint4*)Rx + lane + 32 * k);
        };
        if (kAhead && v < vhi) fetch(v, mask_n, rv_n);
        for (; v < vhi; v += kPairWarps) {
            uint32_t mask;
            uint4 rv[KW];
            if (kAhead) {
                mask = mask_n;
#pragma unroll
                for (int k = 0; k < KW; ++k) rv[k] = rv_n[k];
                if (v + kPairWarps < vhi) fetch(v + kPairWarps, mask_n, rv_n);
            } else {
                fetch(v, mask, rv);
            }
            if (UB == 16) mask = (mask >> ush) & 0xffffu;
            if (v < u0 + UB) mask &= (1u << (int)(v - u0)) - 1u;   // only u < v
            if (!mask) continue;
            const int vw = (int)(v >> 5);
            const uint32_t below_v = (1u << (v & 31)) - 1u;
            uint32_t vsum = 0, myT = 0;   // myT: T(u0 + lane, v) for this lane's u
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint4* ru = (const uint4*)(Rs + b * W);
                const uint32_t T = __reduce_add_sync(0xffffffffu, and_popc<KW>(ru, rv, lane));
                vsum += T;
                if (lane == b) myT = T;
            }
            // the edges of this v with T > 0, one lane each: the per-vertex
            // sum at u, and the flag of (u, v) at its tail position — v's
            // place in N_H(u) — as fire-and-forget updates
            if (myT) {
                const int64_t u = u0 + lane;
                atomicAdd(&Su[lane], myT);
                const int uiw = (int)(u >> 5);
                const uint32_t gt = vw > uiw ? 0xffffffffu : ~((2u << (u & 31)) - 1u);
                const int64_t pos = Hs[lane] + Ps[lane * W + vw] + __popc(Rs[lane * W + vw] & below_v & gt);
                if (ecnt) atomicAdd(&ecnt[TC_IX(pos, dm.e2)], myT);
                else atomicOr(&flag[TC_IX(pos >> 5, dm.fw)], 1u << (pos & 31));
            }
            if (lane == 0 && vsum) {
                atomicAdd(&S[TC_IX(v, C)], (ull)vsum);
                all += vsum;
            }
        }
        __syncthreads();
        if (threadIdx.x < nrows && Su[threadIdx.x]) atomicAdd(&S[u0 + threadIdx.x], (ull)Su[threadIdx.x]);
    }
    if (lane == 0 && all) atomicAdd(sum_t, all);
}

__global__ void k_core_finish(ull* __restrict__ tri, const ull* __restrict__ S, int64_t t, int64_t C,
                              const ull* __restrict__ sum_t, ull* __restrict__ total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x)
        tri[t + i] += S[i] >> 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(total, *sum_t / 3);
}

template <int KW>
tc_status launch_pairs(const uint32_t* R, const uint16_t* P, const tc_graph* g, int64_t t, int64_t C, ull* cursor,
                       ull* S, uint32_t* flag, uint32_t* ecnt, ull* sum_t, cudaStream_t s) {
    constexpr int64_t W = 128 * KW;
    const int ub = core_ub(W);
    const size_t smem = pair_smem(W);
    static std::mutex mu;
    static int per_sm = 0;   // one value per instantiation, set on first use
    {
        std::lock_guard<std::mutex> lk(mu);
        if (per_sm == 0) {
            TC_CUDA(cudaFuncSetAttribute(k_core_pairs<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int b = 0;
            TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_core_pairs<KW>, kPairThreads, smem));
            per_sm = std::max(b, 1);
        }
    }
    const int64_t nblk = (C + ub - 1) / ub, nvch = (C + kVChunk - 1) / kVChunk;
    const int64_t nitems = nblk * nvch;
    const int blocks = (int)std::min<int64_t>((int64_t)sm_count() * per_sm, nitems);
    launch_scope ls("count_core_pairs", s);
    k_core_pairs<KW><<<blocks, kPairThreads, smem, s>>>(R, P, g->hstart, t, C, nvch, nitems, cursor, S, flag, ecnt,
                                                       sum_t, dims_of(g));
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

// Word ANDs of one core pass: every core edge (both ends among the top C
// ranks, i.e. every higher neighbour of a core vertex) ANDs two rows of W words.
double core_word_ops(int64_t C, double core_edges) { return core_edges * (double)core_words(C); }

tc_status core_setup(tc_graph* g, const int32_t* dh, uint32_t flags, cudaStream_t s) {
    g->core_c = 0;
    g->stats.core_vertices = 0;
    g->stats.core_words = 0;
    const long long mode = g_core_mode.load();
    const int64_t n = g->n;
    if (mode == 0 || (flags & TC_BUILD_NO_CORE) || n < 3 || g->m == 0) return TC_OK;
    const int64_t top = std::min<int64_t>(n, mode > 0 ? (int64_t)mode : kCoreMax);
    std::vector<int32_t> h(top);
    TC_CUDA(cudaMemcpyAsync(h.data(), dh + (n - top), top * 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    // edges and wedges of the top c ranks: every higher neighbour of a core
    // vertex is in the core, so its edges number Σ d_H and the ids its rows
    // would stream Σ C(d_H, 2)
    auto sums = [&](int64_t c, double& edges, double& wedges) {
        edges = wedges = 0;
        for (int64_t i = top - c; i < top; ++i) {
            edges += (double)h[i];
            wedges += 0.5 * (double)h[i] * (double)(h[i] - 1);
        }
    };
    int64_t C = 0;
    double E = 0, wdg = 0;
    if (mode > 0) {
        C = top;
        sums(C, E, wdg);
    } else {
        double best = kMinGainMs;
        for (int c : kCoreSizes) {
            if (c > n) break;
            double e = 0, w = 0;
            sums(c, e, w);
            const double cost = core_word_ops(c, e) / kWordsPerMs + kFixedMs;
            const double gain = w / kStreamIdsPerMs - cost;
            if (gain > best) {
                best = gain;
                C = c;
                E = e;
            }
        }
    }
    if (C >= 3) {
        g->core_c = C;
        g->stats.core_vertices = C;
        g->stats.core_words = core_word_ops(C, E);
    }
    return TC_OK;
}

tc_status run_core(tc_graph* g, cudaStream_t s, bool edge_counts) {
    const int64_t C = g->core_c, t = g->n - C;
    if (C <= 0) return TC_OK;
    const int64_t W = core_words(C);
    uint32_t* R = nullptr;
    uint16_t* P = nullptr;
    ull* S = nullptr;
    TC_TRY(dalloc((void**)&R, (size_t)C * W * 4, s));
    tc_status st = dalloc((void**)&P, (size_t)C * W * 2, s);
    if (st == TC_OK) st = dalloc((void**)&S, (size_t)(C + 1) * 8, s);
    if (st == TC_OK) {
        st = [&]() -> tc_status {
            TC_CUDA(cudaMemsetAsync(S, 0, (size_t)(C + 1) * 8, s));
            ull* cursor = g->counters + 6;
            TC_CUDA(cudaMemsetAsync(cursor, 0, 8, s));
            TC_CUDA(cudaMemsetAsync(R, 0, (size_t)C * W * 4, s));
            {
                launch_scope ls("count_core_fill", s);
                const int per = kFillThreads / 32;
                const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((C + per - 1) / per, (int64_t)sm_count() * 8));
                const size_t smem = (size_t)per * W * 4;
                if (smem > 48 * 1024)
                    TC_CUDA(cudaFuncSetAttribute(k_core_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                k_core_fill<<<blocks, kFillThreads, smem, s>>>(g->row_ptr, g->hstart, g->col, t, C, W, R, P, dims_of(g));
                TC_LAUNCH_CHECK();
            }
            uint32_t* ec = edge_counts ? g->ecnt : nullptr;
            switch (W) {
                case 128: TC_TRY(launch_pairs<1>(R, P, g, t, C, cursor, S, g->flag, ec, S + C, s)); break;
                case 256: TC_TRY(launch_pairs<2>(R, P, g, t, C, cursor, S, g->flag, ec, S + C, s)); break;
                case 512: TC_TRY(launch_pairs<4>(R, P, g, t, C, cursor, S, g->flag, ec, S + C, s)); break;
                default: TC_TRY(launch_pairs<8>(R, P, g, t, C, cursor, S, g->flag, ec, S + C, s)); break;
            }
            {
                launch_scope ls("count_core_finish", s);
                const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((C + 255) / 256, (int64_t)sm_count() * 4));
                k_core_finish<<<blocks, 256, 0, s>>>(g->tri, S, t, C, S + C, &g->counters[0]);
                TC_LAUNCH_CHECK();
            }
            return TC_OK;
        }();
    }
    if (S) dfree(S, s);
    if (P) dfree(P, s);
    dfree(R, s);
    return st;
}

}  // namespace tcx

extern "C" tc_status tc_set_dense_core(long long c) {
    if (c < -1 || c > tcx::kCoreMax) return TC_ERR_INVALID_ARG;
    tcx::g_core_mode.store(c);
    return TC_OK;
}
