// tc_build_csr: simple undirected graph, degree order π, orientation and
// the count-step plan, all on the device.
//
//  1. pairs -> canonical keys (min, max); self-loops become a sentinel
//     (the set-up of section "Comparison": symmetrised, loop-free, simple)
//  2. radix sort + unique -> the m undirected edges, caller labels
//  3. degrees; π = sort by (degree, label) (section "Notation")
//  4. every edge relabelled by π and placed in the run of its lower end;
//     each run sorted (warp registers, a warp's shared region or a CTA,
//     by length) -> symmetric CSR in rank space whose rows are
//     [N_L(v) | N_H(v)] (Lemma 1's partition), N_H(v) ascending
//  5. written with the runs: col, edge_tail, and the head record
//     {u, hrem, twin} of every lower neighbour
//  6. planner: per middle vertex v its work W(v) = Σ_{u∈N_L(v)} hrem, and
//     the work items of the count step, heavy vertices split into chunks
//
// Radix sorts (steps 2-3) and scans use CUB (header-only, compiled into
// this library); the per-row run sorts are this file's own.
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
// ranks of its ends, at its canonical id; d_H(lo) counted.
__global__ void k_edge_rank_keys(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                 const int32_t* __restrict__ rank, int64_t m, int bits,
                                 uint64_t* __restrict__ keys, int32_t* __restrict__ dh) {
    GRID_STRIDE(e, m) {
        const uint64_t ru = (uint64_t)rank[eu[e]], rv = (uint64_t)rank[ev[e]];
        const uint64_t lo = ru < rv ? ru : rv, hi = ru < rv ? rv : ru;
        keys[e] = (lo << bits) | hi;
        atomicAdd(&dh[lo], 1);
    }
}

// Row split: the last d_H(r) entries of row r hold N_H(r).  The head cursor
// of row r starts at its first entry (an absolute CSR position), its
// tail-run cursor at hptr[r] (the run's start in the compact tail order).
template <class C>
__global__ void k_hstart(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ dh,
                         const int64_t* __restrict__ hptr, int64_t n, int64_t* __restrict__ hstart,
                         C* __restrict__ hnext, C* __restrict__ tnext) {
    GRID_STRIDE(r, n) {
        hstart[r] = row_ptr[r + 1] - dh[r];
        hnext[r] = (C)row_ptr[r];
        tnext[r] = (C)hptr[r];
    }
}

// Each edge to the next free slot of its lower end's run (row r's run
// starts at hptr[r]) as (hi << 32) | edge id, so that sorting each run puts
// N_H(lo) in order with the edge ids alongside.
template <class C>
__global__ void k_tail_place(const uint64_t* __restrict__ keys, int64_t m, int bits, C* __restrict__ tnext,
                             uint64_t* __restrict__ slot) {
    const uint64_t mask = (1ull << bits) - 1;
    GRID_STRIDE(e, m) {
        const uint64_t k = keys[e];
        const uint64_t lo = k >> bits, hi = k & mask;
        const int64_t i = (int64_t)atomicAdd(&tnext[lo], (C)1);
        slot[i] = (hi << 32) | (uint64_t)e;
    }
}

// Both entries of one edge, from the i-th element x of row r's sorted run
// (tail position t = hstart[r] + i): the tail entry col[t] = hi, the edge's
// canonical id -> t, and the head entry in row hi (N_L(hi) in any order) at
// the next free slot of its cursor, as the record
// {r, |{w ∈ N_H(r) : w > hi}| = e - t - 1, twin = t}.
__device__ __forceinline__ void write_tail(int64_t r, int64_t t, int64_t e, uint64_t x, int64_t hp,
                                           int32_t* __restrict__ col, tc_head* __restrict__ head,
                                           int64_t* __restrict__ edge_tail, int64_t core_t) {
    col[t] = (int32_t)(x >> 32);
    edge_tail[x & 0xffffffffull] = t;
    tc_head rec;
    rec.u = (int32_t)r;
    // a lower end in the dense core (ranks >= core_t) streams nothing: the
    // core's product counts those triangles
    rec.hrem = r >= core_t ? 0 : (int32_t)(e - t - 1);
    rec.twin = t;
    head[hp] = rec;   // one 16-byte store
}

template <class C>
__device__ __forceinline__ void emit_tail(int64_t r, int64_t t, int64_t e, uint64_t x, C* __restrict__ hnext,
                                          int32_t* __restrict__ col, tc_head* __restrict__ head,
                                          int64_t* __restrict__ edge_tail, int64_t core_t) {
    const int64_t hp = (int64_t)atomicAdd(&hnext[(int32_t)(x >> 32)], (C)1);
    write_tail(r, t, e, x, hp, col, head, edge_tail, core_t);
}

// Short runs handled together by one warp in k_runs_small.
constexpr int kSmallGroup = 8;

// Every run is sorted by bitonic merges in the form whose compare-exchanges
// all put the smaller key at the lower index: the first step of the k-merge
// pairs i with its mirror in the k-block (i ^ (k - 1)), the later steps pair
// i with i ^ j.  A run of length L sorts as if padded with +inf up to a
// power of two, since every pair whose upper index is >= L is a no-op; no
// padding is stored.
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t x, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

// One step (merge k, distance j) of the network over key[0, len), padded to
// P, by the threads t0, t0 + nt, ... of a team.
__device__ __forceinline__ void run_network_step(uint64_t* key, int len, int P, int k, int j, int t0, int nt) {
    const int lj = __ffs(j) - 1;
    for (int t = t0; t < (P >> 1); t += nt) {
        const int a = ((t >> lj) << (lj + 1)) | (t & (j - 1));
        const int b = j == (k >> 1) ? a ^ (k - 1) : a | j;
        if (b < len) {
            const uint64_t xa = key[a], xb = key[b];
            if (xb < xa) {
                key[a] = xb;
                key[b] = xa;
            }
        }
    }
}

// Runs of 33..kMidShort tails are sorted by one warp, kMidShort+1..kMidRun
// by one CTA of kMidWarps warps, longer ones by a CTA in shared memory (or
// in place); the first two in registers (below), with the shared-memory
// networks of k_runs_mid kept as the alternative.
constexpr int kMidRun = 1024;
#ifndef TC_MID_SHORT
#define TC_MID_SHORT 256
#endif
constexpr int kMidShort = TC_MID_SHORT;   // longest run of the one-warp tier (512 spilled: slower)

// Runs of 1..32 tails.  A warp takes 32 rows at a time, one per lane:
// single-tail rows are written at once, runs of 2..32 are sorted across the
// warp's registers (keys in lanes 0..L-1, +inf above), kSmallGroup runs at
// a time with the network sized to the longest of them.
// Longer runs are queued: 33..kMidShort tails from the front of `big`
// (count nbig[0]) and kMidShort+1..kMidRun tails from the back of its first
// n entries (count nbig[1]) for k_runs_mid, which never meet since there are
// at most n runs; more than kMidRun tails after those n entries for
// k_runs_big (count nbig[2], fewer than m / kMidRun).
template <class C>
__global__ void k_runs_small(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                             const int64_t* __restrict__ hptr, const uint64_t* __restrict__ slot, int64_t n,
                             C* __restrict__ hnext, int32_t* __restrict__ col, tc_head* __restrict__ head,
                             int64_t* __restrict__ edge_tail, int32_t* __restrict__ big,
                             unsigned int* __restrict__ nbig, int64_t core_t) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += warps * 32) {
        const int64_t r = base + lane;
        int64_t L = 0, p0 = 0, hs = 0, re = 0;
        if (r < n) {
            p0 = hptr[r];
            L = hptr[r + 1] - p0;
            if (L >= 1 && L <= 32) {
                hs = hstart[r];
                re = row_ptr[r + 1];
            }
            if (L == 1) emit_tail(r, hs, re, slot[p0], hnext, col, head, edge_tail, core_t);
            else if (L > kMidRun) big[n + (int64_t)atomicAdd(&nbig[2], 1u)] = (int32_t)r;
            else if (L > kMidShort) big[n - 1 - (int64_t)atomicAdd(&nbig[1], 1u)] = (int32_t)r;
            else if (L > 32) big[atomicAdd(&nbig[0], 1u)] = (int32_t)r;
        }
        unsigned todo = __ballot_sync(0xffffffffu, L >= 2 && L <= 32);
        while (todo) {
            // up to V runs at once: their loads, networks (sized to the
            // longest, padded with +inf) and cursor atomics overlap
            constexpr int V = kSmallGroup;
            int js[V], len[V], maxlen = 0;
            uint64_t x[V];
            int64_t h[V], e[V], hp[V];
#pragma unroll
            for (int u = 0; u < V; ++u) {
                js[u] = todo ? __ffs(todo) - 1 : -1;   // the same in every lane
                todo &= todo - 1;
                len[u] = 0;
                x[u] = ~0ull;
                h[u] = e[u] = 0;
                if (js[u] >= 0) {
                    len[u] = __shfl_sync(0xffffffffu, (int)L, js[u]);
                    const int64_t i0 = __shfl_sync(0xffffffffu, p0, js[u]);
                    h[u] = __shfl_sync(0xffffffffu, hs, js[u]);
                    e[u] = __shfl_sync(0xffffffffu, re, js[u]);
                    if (lane < len[u]) x[u] = slot[i0 + lane];
                    maxlen = max(maxlen, len[u]);
                }
            }
            for (int k = 2; k <= 32 && (k >> 1) < maxlen; k <<= 1) {
                const bool low = (lane & (k - 1)) < (k >> 1);
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    const uint64_t y = shfl_xor64(x[u], k - 1);   // mirror step
                    x[u] = low ? (x[u] < y ? x[u] : y) : (x[u] < y ? y : x[u]);
                }
                for (int jj = k >> 2; jj > 0; jj >>= 1) {
                    const bool lo2 = (lane & jj) == 0;
#pragma unroll
                    for (int u = 0; u < V; ++u) {
                        const uint64_t z = shfl_xor64(x[u], jj);
                        x[u] = lo2 ? (x[u] < z ? x[u] : z) : (x[u] < z ? z : x[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < V; ++u)
                if (lane < len[u]) hp[u] = (int64_t)atomicAdd(&hnext[(int32_t)(x[u] >> 32)], (C)1);
#pragma unroll
            for (int u = 0; u < V; ++u)
                if (lane < len[u]) write_tail(base + js[u], h[u] + lane, e[u], x[u], hp[u], col, head, edge_tail, core_t);
        }
    }
}

// Queued runs of 33..kMidShort tails (CAP = kMidShort: nbig[0] of them at
// the front of `big`) or kMidShort+1..kMidRun tails (CAP = kMidRun: nbig[1]
// at the back of its first n entries): one warp per run, the network in the
// warp's own shared region of CAP keys.
constexpr int kMidWarps = 4;

template <class C, int CAP>
__global__ void __launch_bounds__(32 * kMidWarps)
k_runs_mid(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
           const int64_t* __restrict__ hptr, const uint64_t* __restrict__ slot, const int32_t* __restrict__ big,
           const unsigned int* __restrict__ nbig, int64_t n, C* __restrict__ hnext, int32_t* __restrict__ col,
           tc_head* __restrict__ head, int64_t* __restrict__ edge_tail, int64_t core_t) {
    static_assert(CAP == kMidShort || CAP == kMidRun, "one queue per capacity");
    static_assert(kMidShort == 256 || kMidShort == 512, "register sort tiers: up to 16 keys a lane");
    constexpr bool kBack = CAP == kMidRun;
    __shared__ uint64_t sk[kMidWarps][CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t* key = sk[w];
    const unsigned count = nbig[kBack ? 1 : 0];
    const unsigned warps = gridDim.x * kMidWarps;
    for (unsigned q = blockIdx.x * kMidWarps + w; q < count; q += warps) {
        const int64_t r = kBack ? big[n - 1 - (int64_t)q] : big[q];
        const int64_t i0 = hptr[r];
        const int len = (int)(hptr[r + 1] - i0);
        for (int i = lane; i < len; i += 32) key[i] = slot[i0 + i];
        __syncwarp();
        int P = 1;
        while (P < len) P <<= 1;
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                run_network_step(key, len, P, k, j, lane, 32);
                __syncwarp();
            }
        const int64_t h = hstart[r], e = row_ptr[r + 1];
        for (int i = lane; i < len; i += 32) emit_tail(r, h + i, e, key[i], hnext, col, head, edge_tail, core_t);
        __syncwarp();
    }
}

// Runs of 33..kMidShort tails sorted in registers instead (TC_RUNS_REG):
// key i of the run (i = 32 e + lane, e < E) in register e of a lane, padded
// with +inf to 32 E.  Compare-exchanges at distance j < 32 pair lanes
// (shuffles), at j >= 32 pair registers of one lane; the mirror step of a
// k-merge pairs i with i ^ (k - 1), i.e. lane ^ (k - 1) for k <= 32 and
// register e ^ ((k - 1) >> 5) of lane ^ 31 above.  Loads and the emit's
// col stores are coalesced (lane-consecutive), and no shared memory is used.
#ifndef TC_RUNS_REG
#define TC_RUNS_REG 1
#endif
template <int E>
__device__ __forceinline__ void sort_run_regs(uint64_t (&x)[E], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
        if (k <= 32) {
            const bool low = (lane & (k >> 1)) == 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint64_t y = shfl_xor64(x[e], k - 1);
                x[e] = low ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
            }
        } else {
            // registers e (lower half of the k-block) and f = e ^ m pair with
            // each other's values in lane ^ 31
            const int m = (k - 1) >> 5;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int f = e ^ m;
                if (e < f) {
                    const uint64_t a = shfl_xor64(x[f], 31), b = shfl_xor64(x[e], 31);
                    x[e] = x[e] < a ? x[e] : a;   // e has bit k/64 clear: the lower index
                    x[f] = x[f] < b ? b : x[f];
                }
            }
        }
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
            if (j < 32) {
                const bool low = (lane & j) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint64_t y = shfl_xor64(x[e], j);
                    x[e] = low ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
                }
            } else {
                const int je = j >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((e & je) == 0) {
                        const uint64_t a = x[e], b = x[e | je];
                        x[e] = a < b ? a : b;
                        x[e | je] = a < b ? b : a;
                    }
            }
        }
    }
}

template <class C, int E>
__device__ __forceinline__ void run_regs(int lane, int64_t r, int64_t i0, int len, const uint64_t* __restrict__ slot,
                                         int64_t h, int64_t end, C* __restrict__ hnext, int32_t* __restrict__ col,
                                         tc_head* __restrict__ head, int64_t* __restrict__ edge_tail, int64_t core_t) {
    uint64_t x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = 32 * e + lane;
        x[e] = i < len ? slot[i0 + i] : ~0ull;
    }
    sort_run_regs<E>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = 32 * e + lane;
        if (i < len) emit_tail(r, h + i, end, x[e], hnext, col, head, edge_tail, core_t);
    }
}

template <class C>
__global__ void __launch_bounds__(32 * kMidWarps)
k_runs_mid_reg(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
               const int64_t* __restrict__ hptr, const uint64_t* __restrict__ slot, const int32_t* __restrict__ big,
               const unsigned int* __restrict__ nbig, C* __restrict__ hnext, int32_t* __restrict__ col,
               tc_head* __restrict__ head, int64_t* __restrict__ edge_tail, int64_t core_t) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned count = nbig[0];
    const unsigned warps = gridDim.x * kMidWarps;
    for (unsigned q = blockIdx.x * kMidWarps + w; q < count; q += warps) {
        const int64_t r = big[q];
        const int64_t i0 = hptr[r];
        const int len = (int)(hptr[r + 1] - i0);
        const int64_t h = hstart[r], end = row_ptr[r + 1];
        if (len <= 64) run_regs<C, 2>(lane, r, i0, len, slot, h, end, hnext, col, head, edge_tail, core_t);
        else if (len <= 128) run_regs<C, 4>(lane, r, i0, len, slot, h, end, hnext, col, head, edge_tail, core_t);
        else if (kMidShort <= 256 || len <= 256) run_regs<C, 8>(lane, r, i0, len, slot, h, end, hnext, col, head, edge_tail, core_t);
        else run_regs<C, (kMidShort > 256 ? 16 : 8)>(lane, r, i0, len, slot, h, end, hnext, col, head, edge_tail, core_t);
    }
}

// Runs of kMidShort+1..kMidRun tails by one CTA of kMidWarps warps in
// registers (TC_RUNS_CTA_REG): key i = 32 E w + 32 e + lane in register e of
// lane `lane` of warp w, padded with +inf to 128 E.  Distances below 32 pair
// lanes (shuffles), 32..32E-1 registers of one lane, 32E and above warps,
// through one shared exchange of all keys per such step.
#ifndef TC_RUNS_CTA_REG
#define TC_RUNS_CTA_REG 1
#endif
template <int E>
__device__ __forceinline__ void sort_run_cta(uint64_t (&x)[E], uint64_t* sx, int lane, int w) {
    constexpr int P = 32 * E * kMidWarps;
    const int me = 32 * E * w + lane;   // index of register 0
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
        if (k <= 32) {
            const bool low = (lane & (k >> 1)) == 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint64_t y = shfl_xor64(x[e], k - 1);
                x[e] = low ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
            }
        } else if (k <= 32 * E) {
            const int m = (k - 1) >> 5;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int f = e ^ m;
                if (e < f) {
                    const uint64_t a = shfl_xor64(x[f], 31), b = shfl_xor64(x[e], 31);
                    x[e] = x[e] < a ? x[e] : a;
                    x[f] = x[f] < b ? b : x[f];
                }
            }
        } else {
            // partner of i is i ^ (k - 1): another warp, register E-1-e, lane ^ 31
#pragma unroll
            for (int e = 0; e < E; ++e) sx[me + 32 * e] = x[e];
            __syncthreads();
            const int pw = w ^ ((k - 1) / (32 * E));
            const bool low = (w & (k / (64 * E))) == 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint64_t y = sx[32 * E * pw + 32 * (E - 1 - e) + (lane ^ 31)];
                x[e] = low ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
            if (j < 32) {
                const bool low = (lane & j) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint64_t y = shfl_xor64(x[e], j);
                    x[e] = low ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
                }
            } else if (j < 32 * E) {
                const int je = j >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((e & je) == 0) {
                        const uint64_t a = x[e], b = x[e | je];
                        x[e] = a < b ? a : b;
                        x[e | je] = a < b ? b : a;
                    }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) sx[me + 32 * e] = x[e];
                __syncthreads();
                const int pw = w ^ (j / (32 * E));
                const bool low = (w & (j / (32 * E))) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint64_t y = sx[32 * E * pw + 32 * e + lane];
                    x[e] = low ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
                }
                __syncthreads();
            }
        }
    }
}

template <class C, int E>
__device__ __forceinline__ void run_cta(int lane, int w, uint64_t* sx, int64_t r, int64_t i0, int len,
                                        const uint64_t* __restrict__ slot, int64_t h, int64_t end,
                                        C* __restrict__ hnext, int32_t* __restrict__ col,
                                        tc_head* __restrict__ head, int64_t* __restrict__ edge_tail, int64_t core_t) {
    uint64_t x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = 32 * E * w + 32 * e + lane;
        x[e] = i < len ? slot[i0 + i] : ~0ull;
    }
    sort_run_cta<E>(x, sx, lane, w);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = 32 * E * w + 32 * e + lane;
        if (i < len) emit_tail(r, h + i, end, x[e], hnext, col, head, edge_tail, core_t);
    }
}

template <class C>
__global__ void __launch_bounds__(32 * kMidWarps)
k_runs_long_cta(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                const int64_t* __restrict__ hptr, const uint64_t* __restrict__ slot, const int32_t* __restrict__ big,
                const unsigned int* __restrict__ nbig, int64_t n, C* __restrict__ hnext, int32_t* __restrict__ col,
                tc_head* __restrict__ head, int64_t* __restrict__ edge_tail, int64_t core_t) {
    static_assert(32 * 8 * kMidWarps == kMidRun, "eight keys a thread cover the longest queued run");
    __shared__ uint64_t sx[kMidRun];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned count = nbig[1];
    for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
        const int64_t r = big[n - 1 - (int64_t)q];
        const int64_t i0 = hptr[r];
        const int len = (int)(hptr[r + 1] - i0);
        const int64_t h = hstart[r], end = row_ptr[r + 1];
        if (len <= 512) run_cta<C, 4>(lane, w, sx, r, i0, len, slot, h, end, hnext, col, head, edge_tail, core_t);
        else run_cta<C, 8>(lane, w, sx, r, i0, len, slot, h, end, hnext, col, head, edge_tail, core_t);
    }
}

// Queued runs longer than kMidRun (nbig[2] of them, after the first n
// entries of `big`): one CTA per run, the network in shared memory (up to
// kRunSmem keys) or in place in `slot`.
constexpr int kRunSmem = 4096;
constexpr int kRunThreads = 512;

template <class C>
__global__ void __launch_bounds__(kRunThreads)
k_runs_big(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
           const int64_t* __restrict__ hptr, uint64_t* __restrict__ slot, const int32_t* __restrict__ big,
           const unsigned int* __restrict__ nbig, int64_t n, C* __restrict__ hnext, int32_t* __restrict__ col,
           tc_head* __restrict__ head, int64_t* __restrict__ edge_tail, int64_t core_t) {
    __shared__ uint64_t sk[kRunSmem];
    const unsigned count = nbig[2];
    for (unsigned q = blockIdx.x; q < count; q += gridDim.x) {
        const int64_t r = big[n + (int64_t)q];
        const int64_t i0 = hptr[r];
        const int len = (int)(hptr[r + 1] - i0);
        uint64_t* key = len <= kRunSmem ? sk : slot + i0;
        if (len <= kRunSmem)
            for (int i = threadIdx.x; i < len; i += blockDim.x) sk[i] = slot[i0 + i];
        __syncthreads();
        int P = 1;
        while (P < len) P <<= 1;
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                run_network_step(key, len, P, k, j, threadIdx.x, blockDim.x);
                __syncthreads();
            }
        const int64_t h = hstart[r], e = row_ptr[r + 1];
        for (int i = threadIdx.x; i < len; i += blockDim.x) emit_tail(r, h + i, e, key[i], hnext, col, head, edge_tail, core_t);
        __syncthreads();
    }
}

// First ranks whose degree exceeds 32 and TC_BAND_CTA (degrees ascend with
// rank): the gather and the per-row work take one thread, one warp and one
// CTA per row in the three bands.
#ifndef TC_BAND_CTA
#define TC_BAND_CTA 4096
#endif
__global__ void k_bands(const int64_t* __restrict__ row_ptr, int64_t n, int64_t* __restrict__ band) {
    const int64_t lim[2] = {32, TC_BAND_CTA};
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

// W(v) = Σ_{u ∈ N_L(v)} hrem(u, v), the number of ids the count step
// streams for middle vertex v, plus shape statistics.  Rows ascend in
// degree: rows below band[0] (degree <= 32) take one thread each, the rest
// one warp each.
// Rows of degree above 4096 get one CTA each in the per-row work (below).
#ifndef TC_ROW_WORK_CTA
#define TC_ROW_WORK_CTA 1
#endif
struct row_acc {
    unsigned long long h2 = 0, w = 0, dh = 0, maxh = 0, maxd = 0;
    __device__ __forceinline__ void add(unsigned long long hv, unsigned long long d, unsigned long long wr) {
        h2 += hv * hv;
        w += wr;
        dh += d * hv;
        maxh = maxh > hv ? maxh : hv;
        maxd = maxd > d ? maxd : d;
    }
    __device__ __forceinline__ void flush(row_stats* st) {
        for (int o = 16; o; o >>= 1) {
            h2 += __shfl_xor_sync(0xffffffffu, h2, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
            dh += __shfl_xor_sync(0xffffffffu, dh, o);
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, maxh, o);
            const unsigned long long c = __shfl_xor_sync(0xffffffffu, maxd, o);
            maxh = maxh > a ? maxh : a;
            maxd = maxd > c ? maxd : c;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&st->sum_h2, h2);
            atomicAdd(&st->wedges, w);
            atomicAdd(&st->sum_dh, dh);
            atomicMax(&st->max_h, maxh);
            atomicMax(&st->max_d, maxd);
        }
    }
};

__global__ void k_row_work_thread(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                                  const tc_head* __restrict__ head, const int64_t* __restrict__ band,
                                  int64_t* __restrict__ work, row_stats* __restrict__ st) {
    const int64_t r1 = band[0];
    row_acc acc;
    // whole warps step together so that the final shuffles see every lane
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp_first = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll;
    for (int64_t base = warp_first; base < r1; base += stride) {
        const int64_t r = base + (threadIdx.x & 31);
        if (r < r1) {
            const int64_t b = row_ptr[r], h = hstart[r], e = row_ptr[r + 1];
            unsigned long long w = 0;
            for (int64_t p = b; p < h; ++p) w += (unsigned long long)head[p].hrem;
            work[r] = (int64_t)w;
            acc.add((unsigned long long)(e - h), (unsigned long long)(e - b), w);
        }
    }
    acc.flush(st);
}

__global__ void k_row_work_warp(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                                const tc_head* __restrict__ head, const int64_t* __restrict__ band, int64_t n,
                                int64_t* __restrict__ work, row_stats* __restrict__ st) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    row_acc acc;
    const int64_t r1 = TC_ROW_WORK_CTA ? band[1] : n;   // rows above degree 4096: k_row_work_cta
    for (int64_t r = band[0] + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); r < r1; r += warps) {
        const int64_t b = row_ptr[r], h = hstart[r], e = row_ptr[r + 1];
        unsigned long long w = 0;
        for (int64_t p = b + lane; p < h; p += 32) w += (unsigned long long)head[p].hrem;
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) {
            work[r] = (int64_t)w;
            acc.add((unsigned long long)(e - h), (unsigned long long)(e - b), w);
        }
    }
    acc.flush(st);
}

// Rows of degree above 4096 (ranks band[1] .. n - 1, the hubs, up to
// hundreds of thousands of head entries each): one CTA per row, so that
// the last hub rows do not each keep a single warp busy after the rest.
__global__ void __launch_bounds__(512) k_row_work_cta(const int64_t* __restrict__ row_ptr,
                                                      const int64_t* __restrict__ hstart,
                                                      const tc_head* __restrict__ head,
                                                      const int64_t* __restrict__ band, int64_t n,
                                                      int64_t* __restrict__ work, row_stats* __restrict__ st) {
    __shared__ unsigned long long part[16];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    row_acc acc;
    for (int64_t r = band[1] + blockIdx.x; r < n; r += gridDim.x) {
        const int64_t b = row_ptr[r], h = hstart[r], e = row_ptr[r + 1];
        unsigned long long w = 0;
        for (int64_t p = b + threadIdx.x; p < h; p += blockDim.x) w += (unsigned long long)head[p].hrem;
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) part[wp] = w;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long s = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
            work[r] = (int64_t)s;
            acc.add((unsigned long long)(e - h), (unsigned long long)(e - b), s);
        }
        __syncthreads();
    }
    acc.flush(st);
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
    // called inside a launch_scope: the sort's own kernels counted beyond it
    const int64_t k = library_kernels("radix_sort_keys", count, end_bit, [&](cudaStream_t p) {
        cub::DoubleBuffer<T> probe = buf;   // the real call flips buf's selector
        return cub::DeviceRadixSort::SortKeys(tmp, bytes, probe, count, 0, end_bit, p);
    });
    TC_CUDA(cub::DeviceRadixSort::SortKeys(tmp, bytes, buf, count, 0, end_bit, s));
    add_launches(k - 1);
    return TC_OK;
}

// Step 4 after the run offsets: row split and cursors, tail placement,
// then the runs sorted and written by length class.
template <class C>
tc_status build_runs(tc_graph* g, cudaStream_t s, int64_t m, int64_t n, int bits, const uint64_t* keys,
                     uint64_t* slot, const int32_t* dh, const int64_t* hptr, int32_t* big, unsigned int* nbig,
                     C* hnext, C* tnext, int rows_blocks, int64_t core_t) {
    {
        launch_scope ls("build_hstart", s);
        k_hstart<<<grid_for(n), kThreads, 0, s>>>(g->row_ptr, dh, hptr, n, g->hstart, hnext, tnext);
        TC_LAUNCH_CHECK();
    }
    {
        launch_scope ls("build_tail_place", s);
        k_tail_place<<<grid_for(m), kThreads, 0, s>>>(keys, m, bits, tnext, slot);
        TC_LAUNCH_CHECK();
    }
    {
        launch_scope ls("build_runs_small", s);
        k_runs_small<<<rows_blocks, kThreads, 0, s>>>(g->row_ptr, g->hstart, hptr, slot, n, hnext, g->col,
                                                      g->head, g->edge_tail, big, nbig, core_t);
        TC_LAUNCH_CHECK();
    }
    {
        launch_scope ls("build_runs_mid", s);
        if (TC_RUNS_REG)
            k_runs_mid_reg<C><<<sm_count() * 16, 32 * kMidWarps, 0, s>>>(
                g->row_ptr, g->hstart, hptr, slot, big, nbig, hnext, g->col, g->head, g->edge_tail, core_t);
        else
            k_runs_mid<C, kMidShort><<<sm_count() * 16, 32 * kMidWarps, 0, s>>>(
                g->row_ptr, g->hstart, hptr, slot, big, nbig, n, hnext, g->col, g->head, g->edge_tail, core_t);
        TC_LAUNCH_CHECK();
    }
    {
        launch_scope ls("build_runs_long", s);
        if (TC_RUNS_CTA_REG)
            k_runs_long_cta<C><<<sm_count() * 16, 32 * kMidWarps, 0, s>>>(
                g->row_ptr, g->hstart, hptr, slot, big, nbig, n, hnext, g->col, g->head, g->edge_tail, core_t);
        else
            k_runs_mid<C, kMidRun><<<sm_count() * 8, 32 * kMidWarps, 0, s>>>(
                g->row_ptr, g->hstart, hptr, slot, big, nbig, n, hnext, g->col, g->head, g->edge_tail, core_t);
        TC_LAUNCH_CHECK();
    }
    {
        launch_scope ls("build_runs_big", s);
        k_runs_big<<<sm_count() * 2, kRunThreads, 0, s>>>(g->row_ptr, g->hstart, hptr, slot, big, nbig, n,
                                                          hnext, g->col, g->head, g->edge_tail, core_t);
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}

}  // namespace

void free_graph_memory(tc_graph* g) {
    cudaStream_t s = g->stream;
    void* ptrs[] = {g->edge_u, g->edge_v, g->perm, g->row_ptr, g->col, g->hstart, g->head,
                    g->edge_tail, g->work, g->tri, g->flag, g->tri32, g->counters, g->ecnt};
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
        copy_scope cs("copy_h2d_pairs", s);
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
            TC_TRY(run_library("select_unique", np, 0, true, s, [&](cudaStream_t st) {
                return cub::DeviceSelect::Unique(tmp, bytes, sorted, uniq, d_nsel, np, st);
            }));
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
    TC_TRY(dalloc((void**)&g->tri32, (n + 1) * 4, s));
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
        // the sort key is (degree << bits | label): it needs only as many
        // degree bits as the largest degree has
        int32_t* d_maxdeg = nullptr;
        TC_TRY(sc.get(&d_maxdeg, 1));
        size_t rbytes = 0;
        TC_CUDA(cub::DeviceReduce::Max(nullptr, rbytes, deg, d_maxdeg, n, s));
        uint8_t* rtmp = nullptr;
        TC_TRY(sc.get(&rtmp, rbytes));
        {
            launch_scope ls("build_max_degree", s);
            TC_TRY(run_library("reduce_max", n, 0, true, s, [&](cudaStream_t st) {
                return cub::DeviceReduce::Max(rtmp, rbytes, deg, d_maxdeg, n, st);
            }));
        }
        int32_t maxdeg = 0;
        TC_CUDA(cudaMemcpyAsync(&maxdeg, d_maxdeg, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        cub::DoubleBuffer<uint64_t> rbuf(ra, rb);
        {
            launch_scope ls("build_sort_rank", s);
            TC_TRY(sort_keys(sc, rbuf, n, bits + bits_for((int64_t)maxdeg + 1), s));
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
        TC_TRY(run_library("scan_i64", n + 1, 0, true, s, [&](cudaStream_t st) {
            return cub::DeviceScan::ExclusiveSum(tmp, bytes, degr, g->row_ptr, n + 1, st);
        }));
    }

    // ---- 4. rank-space CSR: every edge placed in its lower end's run of
    // tails, each run sorted (N_H(r) ascending) and both entries written;
    // the heads N_L(r) need no order
    if (m > 0) {
        uint64_t *keys = nullptr, *slot = nullptr;
        int32_t *dh = nullptr, *big = nullptr;
        unsigned int* nbig = nullptr;
        void* hnext = nullptr;   // head cursors (absolute positions)
        void* tnext = nullptr;   // tail-run cursors (compact order)
        int64_t* hptr = nullptr;
        const bool narrow = e2 < ((int64_t)1 << 32);   // 32-bit cursors suffice
        TC_TRY(sc.get(&keys, m));
        TC_TRY(sc.get(&slot, m));
        TC_TRY(sc.get(&dh, n + 1));
        TC_TRY(sc.get(&big, n + m / kMidRun + 2));
        TC_TRY(sc.get(&nbig, 3));
        TC_TRY(sc.get((uint8_t**)&hnext, (n + 1) * (narrow ? 4 : 8)));
        TC_TRY(sc.get((uint8_t**)&tnext, (n + 1) * (narrow ? 4 : 8)));
        TC_TRY(sc.get(&hptr, n + 1));
        TC_CUDA(cudaMemsetAsync(dh, 0, (n + 1) * 4, s));
        TC_CUDA(cudaMemsetAsync(nbig, 0, 3 * sizeof(unsigned int), s));
        {
            launch_scope ls("build_edge_rank_keys", s);
            k_edge_rank_keys<<<grid_for(m), kThreads, 0, s>>>(g->edge_u, g->edge_v, rank, m, bits, keys, dh);
            TC_LAUNCH_CHECK();
        }
        size_t sbytes = 0;
        TC_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, sbytes, dh, hptr, n + 1, s));
        uint8_t* tmp = nullptr;
        TC_TRY(sc.get(&tmp, sbytes));
        {
            launch_scope ls("build_hptr", s);
            TC_TRY(run_library("scan_i32", n + 1, 0, true, s, [&](cudaStream_t st) {
                return cub::DeviceScan::ExclusiveSum(tmp, sbytes, dh, hptr, n + 1, st);
            }));
        }
        const int cap = sm_count() * 16;
        const int rows_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, cap));
        // the dense core, if one pays: its rows' head records stream nothing
        TC_TRY(core_setup(g, dh, flags, s));
        const int64_t core_t = n - g->core_c;
        if (narrow) {
            TC_TRY(build_runs(g, s, m, n, bits, keys, slot, dh, hptr, big, nbig, (uint32_t*)hnext,
                              (uint32_t*)tnext, rows_blocks, core_t));
        } else {
            TC_TRY(build_runs(g, s, m, n, bits, keys, slot, dh, hptr, big, nbig, (unsigned long long*)hnext,
                              (unsigned long long*)tnext, rows_blocks, core_t));
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
    int64_t* d_band = nullptr;
    TC_TRY(sc.get(&d_band, 2));
    {
        launch_scope ls("build_bands", s);
        k_bands<<<1, 1, 0, s>>>(g->row_ptr, n, d_band);
        TC_LAUNCH_CHECK();
    }
    if (n > 0) {
        const int cap = sm_count() * 16;
        {
            launch_scope ls("build_row_work_thread", s);
            const int bt = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)cap);
            k_row_work_thread<<<std::max(bt, 1), kThreads, 0, s>>>(g->row_ptr, g->hstart, g->head, d_band,
                                                                   g->work, dst_stats);
            TC_LAUNCH_CHECK();
        }
        {
            launch_scope ls("build_row_work_warp", s);
            const int bw = (int)std::min<int64_t>((n * 32 + kThreads - 1) / kThreads, (int64_t)cap);
            k_row_work_warp<<<std::max(bw, 1), kThreads, 0, s>>>(g->row_ptr, g->hstart, g->head, d_band, n,
                                                                 g->work, dst_stats);
            TC_LAUNCH_CHECK();
        }
        if (TC_ROW_WORK_CTA) {
            launch_scope ls("build_row_work_cta", s);
            k_row_work_cta<<<sm_count() * 4, 512, 0, s>>>(g->row_ptr, g->hstart, g->head, d_band, n, g->work,
                                                          dst_stats);
            TC_LAUNCH_CHECK();
        }
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
    // (8+8+4+8+8+8) and the 32-bit copy of △(v) made first (8 in, 4 out); per
    // adjacency entry its label and the neighbour's count from that copy
    // (4+4); per head entry twin and the mirrored flag (8+1); per tail entry
    // its flag (1).
    S.centrality_bytes = 56.0 * n + 8.0 * (double)e2 + 9.0 * m + 1.0 * m;
    // Target work of a CTA item: large items stage N_H(v) less often, small
    // ones spread a few heavy vertices over more CTAs.  About 64 items' worth
    // of the graph's wedges per SM, within [2^16, 2^22] (R-MAT scale 24: 2^22;
    // the 4096^2 grid with its Chung-Lu hubs: 2^16, where 2^22 left the
    // bitmap kernel 2.5 times slower).  tc_set_plan_params overrides it.
    {
        const double per = S.wedges / (64.0 * (double)sm_count());
        g->params.cta_chunk = (int64_t)std::min(4194304.0, std::max(65536.0, per));
    }
    // Unions of many small graphs hold millions of light vertices; one
    // thread each for those of up to 128 ids of work instead of 64 (the
    // 8192-graph batch: count 7.9 -> 6.7 ms; on the grid workload the
    // larger cap was 0.3 ms slower, so single graphs keep 64).
    if (flags & TC_BUILD_NO_CORE) g->params.thread_work = 128;
    TC_TRY(make_plan(g, g->strategy, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

}  // namespace tcx
