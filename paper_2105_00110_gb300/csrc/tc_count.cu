// tc_count: triangle counts △(v), △(G) and edge flags (steps 1-2 of the
// elementary algorithm, section "Algorithm").
//
// Orientation as in Procedure 1: every triangle u < v < w (rank order) is
// met exactly once, from its middle vertex v and its lowest vertex u ∈ N_L(v),
// as an id w of N_H(u) that is also in N_H(v).  The count kernels stage
// N_H(v) on chip once per work item (Procedure 1's marker array T, here a
// sorted list, a bitmap or nothing for the global variant) and stream, for
// every lower neighbour u in the item, only the part of N_H(u) above v:
// col[twin(u,v)+1 .. row_end(u)), since ids at or below v cannot be in N_H(v).
//
// A hit (u, v, w) adds one to △(u), △(v), △(w), △(G) and marks the three
// edges as triangle edges.  Flags live on the canonical (tail) entry of each
// edge — the position of the higher end in the lower end's N_H — which is
// the layout of the per-position arrays L_v of the appendix procedure
// ("Alternative Triangle Neighbor Algorithm"): (u,w) at the streamed
// position, (v,w) at the staged position, (u,v) at twin(u,v).
//
// Counts are aggregated on chip before the integer atomics: per staged id
// (shared-memory counters, flushed once per item), per lower neighbour (one
// counter per batch entry), per middle vertex (a register).
#include <algorithm>

#include "tc_internal.cuh"

namespace tcx {

namespace {

enum { MODE_BSEARCH = 0, MODE_MERGE = 1, MODE_BITMAP = 2, MODE_GLOBAL = 3 };

typedef unsigned long long ull;

// Per-warp batch bookkeeping: 32 head entries (lower neighbours u) at a time.
struct batch_smem {
    int64_t start[32];   // first streamed position: twin(u,v) + 1
    int32_t excl[33];    // exclusive prefix of the streamed lengths, [32] = total
    uint32_t hits[32];   // triangles found per entry
};

// Index of w in the ascending list a[0, len), or -1.
__device__ __forceinline__ int find_sorted(const int32_t* a, int len, int32_t w) {
    int lo = 0;
    while (len > 0) {
        int half = len >> 1;
        if (a[lo + half] < w) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;  // caller checks bounds and equality
}

__device__ __forceinline__ int64_t find_sorted_global(const int32_t* __restrict__ a, int64_t len, int32_t w) {
    int64_t lo = 0;
    while (len > 0) {
        int64_t half = len >> 1;
        if (__ldg(a + lo + half) < w) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// The staged N_H(v) of the current item.
struct staged {
    const int32_t* ids;      // ascending ids (shared memory, or global for MODE_GLOBAL)
    int hv;
    uint32_t* cnt;           // per staged index hit counters (shared), unused for MODE_GLOBAL
    const uint32_t* bits;    // MODE_BITMAP: bit (w - base) set iff w ∈ N_H(v)
    const uint32_t* rank;    // MODE_BITMAP: set bits in words before word k
    int32_t base;
    int32_t nbits;
    int64_t h0;              // position of N_H(v) in col
};

// Loads one batch of head entries [b, min(b+32, pe)) into the warp's batch
// bookkeeping and returns the total number of streamed ids in it.
__device__ __forceinline__ int load_batch(int lane, int64_t b, int64_t pe,
                                          const int32_t* __restrict__ col,
                                          const int64_t* __restrict__ twin,
                                          const int32_t* __restrict__ hrem,
                                          batch_smem& bs, int32_t& u, bool& valid) {
    int64_t p = b + lane;
    valid = p < pe;
    int64_t t = 0;
    int r = 0;
    u = 0;
    if (valid) {
        u = col[p];
        t = twin[p];
        r = hrem[p];
    }
    int incl = r;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int x = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += x;
    }
    int total = __shfl_sync(0xffffffffu, incl, 31);
    bs.start[lane] = t + 1;
    bs.excl[lane] = incl - r;
    bs.hits[lane] = 0;
    if (lane == 0) bs.excl[32] = total;
    __syncwarp();
    return total;
}

// Records a hit: triangle (u, v, w) with w found at staged index l and at
// column position pos (inside N_H(u)); s is the batch entry of u.
template <int MODE>
__device__ __forceinline__ void on_hit(const staged& st, batch_smem& bs, int s, int l,
                                       int32_t w, int64_t pos, ull* __restrict__ tri,
                                       uint8_t* __restrict__ flag) {
    if (MODE == MODE_GLOBAL) {
        atomicAdd(&tri[w], 1ull);
        flag[st.h0 + l] = 1;
    } else {
        atomicAdd(&st.cnt[l], 1u);
    }
    atomicAdd(&bs.hits[s], 1u);
    flag[pos] = 1;
}

// Flattened streaming of one batch: lane i takes streamed ids i, i+32, ...
// of the concatenated lists and looks each up in the staged N_H(v).
template <int MODE>
__device__ __forceinline__ void stream_batch(int lane, int total, const staged& st, batch_smem& bs,
                                             const int32_t* __restrict__ col, ull* __restrict__ tri,
                                             uint8_t* __restrict__ flag) {
    for (int f = lane; f < total; f += 32) {
        int s = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1)
            if (bs.excl[s + step] <= f) s += step;
        int64_t pos = bs.start[s] + (f - bs.excl[s]);
        int32_t w = __ldg(col + pos);
        int l;
        bool hit;
        if (MODE == MODE_BITMAP) {
            int32_t off = w - st.base;
            hit = off >= 0 && off < st.nbits;
            l = 0;
            if (hit) {
                uint32_t word = st.bits[off >> 5];
                uint32_t bit = 1u << (off & 31);
                hit = (word & bit) != 0;
                l = (int)st.rank[off >> 5] + __popc(word & (bit - 1));
            }
        } else if (MODE == MODE_GLOBAL) {
            int64_t k = find_sorted_global(st.ids, st.hv, w);
            hit = k < st.hv && __ldg(st.ids + k) == w;
            l = (int)k;
        } else {
            l = find_sorted(st.ids, st.hv, w);
            hit = l < st.hv && st.ids[l] == w;
        }
        if (hit) on_hit<MODE>(st, bs, s, l, w, pos, tri, flag);
    }
}

// Merge-path intersection of the staged A = N_H(v) (shared, ascending) with
// B = col[bstart, bstart + r) for each batch entry in turn.  The 32 lanes
// split the merge path of A and B into equal diagonals; on ties the A
// element is consumed first, and a common id is counted when its A element
// is consumed with the current B element equal to it.
__device__ __forceinline__ void merge_batch(int lane, const staged& st, batch_smem& bs,
                                            const int32_t* __restrict__ col, ull* __restrict__ tri,
                                            uint8_t* __restrict__ flag) {
    const int32_t* A = st.ids;
    const int na = st.hv;
    for (int s = 0; s < 32; ++s) {
        int nb = bs.excl[s + 1] - bs.excl[s];
        if (nb == 0) continue;
        const int32_t* B = col + bs.start[s];
        int L = na + nb;
        int d0 = (int)(((int64_t)L * lane) >> 5), d1 = (int)(((int64_t)L * (lane + 1)) >> 5);
        // i = number of A elements among the first d0 merge steps
        int lo = max(0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (A[mid] <= __ldg(B + (d0 - mid - 1))) lo = mid + 1; else hi = mid;
        }
        int i = lo, j = d0 - lo;
        for (int d = d0; d < d1; ++d) {
            if (i < na && (j >= nb || A[i] <= __ldg(B + j))) {
                if (j < nb && __ldg(B + j) == A[i])
                    on_hit<MODE_MERGE>(st, bs, s, i, A[i], bs.start[s] + j, tri, flag);
                ++i;
            } else {
                ++j;
            }
        }
    }
}

// Credits the hits of a finished batch to △(u) and flags (u, v).
__device__ __forceinline__ void close_batch(int lane, bool valid, int32_t u, batch_smem& bs,
                                            ull* __restrict__ tri, uint8_t* __restrict__ flag,
                                            ull& tv) {
    __syncwarp();
    if (valid) {
        uint32_t c = bs.hits[lane];
        if (c) {
            atomicAdd(&tri[u], (ull)c);
            flag[bs.start[lane] - 1] = 1;   // twin(u, v): the canonical entry of (u, v)
            tv += c;
        }
    }
    __syncwarp();
}

template <int MODE>
__device__ __forceinline__ void run_batches(int lane, int64_t first, int64_t pe, int64_t stride,
                                            const staged& st, batch_smem& bs,
                                            const int32_t* __restrict__ col,
                                            const int64_t* __restrict__ twin,
                                            const int32_t* __restrict__ hrem,
                                            ull* __restrict__ tri, uint8_t* __restrict__ flag,
                                            ull& tv) {
    for (int64_t b = first; b < pe; b += stride) {
        int32_t u;
        bool valid;
        int total = load_batch(lane, b, pe, col, twin, hrem, bs, u, valid);
        if (total > 0) {
            if (MODE == MODE_MERGE) merge_batch(lane, st, bs, col, tri, flag);
            else stream_batch<MODE>(lane, total, st, bs, col, tri, flag);
        }
        close_batch(lane, valid, u, bs, tri, flag, tv);
    }
}

__device__ __forceinline__ ull warp_sum(ull x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ------------------------------------------------------------ warp items
struct warp_smem {
    int32_t ids[TC_WARP_CAP];
    uint32_t cnt[TC_WARP_CAP];
    batch_smem bs;
};

constexpr int kWarpItemsPerFetch = 4;

__global__ void __launch_bounds__(TC_CTA_THREADS)
k_count_warp(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
             const int64_t* __restrict__ hstart, const int64_t* __restrict__ twin,
             const int32_t* __restrict__ hrem, const int32_t* __restrict__ it_v,
             const int64_t* __restrict__ it_pb, const int64_t* __restrict__ it_pe,
             int64_t n_items, ull* __restrict__ cursor, int strategy, ull* __restrict__ tri,
             uint8_t* __restrict__ flag, ull* __restrict__ total) {
    __shared__ warp_smem sm[TC_CTA_THREADS / 32];
    const int lane = threadIdx.x & 31;
    warp_smem& ws = sm[threadIdx.x >> 5];
    const int mode = (strategy == TC_STRATEGY_MERGE) ? MODE_MERGE : MODE_BSEARCH;
    ull tv_all = 0;
    for (;;) {
        int64_t base = 0;
        if (lane == 0) base = (int64_t)atomicAdd(cursor, (ull)kWarpItemsPerFetch);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_items) break;
        int64_t lim = min(base + kWarpItemsPerFetch, n_items);
        for (int64_t it = base; it < lim; ++it) {
            const int32_t v = it_v[it];
            const int64_t pb = it_pb[it], pe = it_pe[it];
            const int64_t h0 = hstart[v];
            const int hv = (int)(row_ptr[v + 1] - h0);
            for (int i = lane; i < hv; i += 32) {
                ws.ids[i] = col[h0 + i];
                ws.cnt[i] = 0;
            }
            __syncwarp();
            staged st{ws.ids, hv, ws.cnt, nullptr, nullptr, 0, 0, h0};
            ull tv = 0;
            if (mode == MODE_MERGE)
                run_batches<MODE_MERGE>(lane, pb, pe, 32, st, ws.bs, col, twin, hrem, tri, flag, tv);
            else
                run_batches<MODE_BSEARCH>(lane, pb, pe, 32, st, ws.bs, col, twin, hrem, tri, flag, tv);
            __syncwarp();
            for (int i = lane; i < hv; i += 32) {
                uint32_t c = ws.cnt[i];
                if (c) {
                    atomicAdd(&tri[ws.ids[i]], (ull)c);
                    flag[h0 + i] = 1;
                }
            }
            tv = warp_sum(tv);
            if (lane == 0 && tv) atomicAdd(&tri[v], tv);
            tv_all += tv;
            __syncwarp();
        }
    }
    if (lane == 0 && tv_all) atomicAdd(total, tv_all);
}

// ------------------------------------------------------------- CTA items
constexpr int kCtaWarps = TC_CTA_THREADS / 32;

__device__ __forceinline__ int cta_mode(int strategy, int hv, int64_t window_bits, int64_t work,
                                        size_t room) {
    const size_t list_bytes = (size_t)hv * 8;                 // ids + counters
    const int64_t words = (window_bits + 31) >> 5;
    const size_t bitmap_bytes = (size_t)words * 8 + (size_t)hv * 4;  // bits + rank + counters
    const bool list_fits = list_bytes <= room;
    const bool bitmap_fits = bitmap_bytes <= room && window_bits < (1ll << 31);
    if (strategy == TC_STRATEGY_BITMAP) return bitmap_fits ? MODE_BITMAP : (list_fits ? MODE_BSEARCH : MODE_GLOBAL);
    if (strategy == TC_STRATEGY_MERGE) return list_fits ? MODE_MERGE : MODE_GLOBAL;
    if (strategy == TC_STRATEGY_BSEARCH) return list_fits ? MODE_BSEARCH : MODE_GLOBAL;
    // AUTO: the bitmap when zeroing it costs little next to the item's work
    if (bitmap_fits && words * 16 <= work) return MODE_BITMAP;
    return list_fits ? MODE_BSEARCH : MODE_GLOBAL;
}

__global__ void __launch_bounds__(TC_CTA_THREADS)
k_count_cta(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
            const int64_t* __restrict__ hstart, const int64_t* __restrict__ twin,
            const int32_t* __restrict__ hrem, const int32_t* __restrict__ it_v,
            const int64_t* __restrict__ it_pb, const int64_t* __restrict__ it_pe,
            int64_t n_items, ull* __restrict__ cursor, int strategy, size_t smem_bytes,
            ull* __restrict__ tri, uint8_t* __restrict__ flag, ull* __restrict__ total) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ batch_smem bsm[kCtaWarps];
    __shared__ int64_t s_item;
    __shared__ ull s_tv[kCtaWarps];
    __shared__ uint32_t s_scan[kCtaWarps + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = blockDim.x;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(cursor, 1ull);
        __syncthreads();
        const int64_t it = s_item;
        if (it >= n_items) break;
        const int32_t v = it_v[it];
        const int64_t pb = it_pb[it], pe = it_pe[it];
        const int64_t h0 = hstart[v], h1 = row_ptr[v + 1];
        const int hv = (int)(h1 - h0);
        int64_t work = 0;  // approximate: head entries x mean remainder is not known; use entries
        work = (pe - pb) * 64;
        const int32_t base = v + 1;
        const int64_t window = (int64_t)col[h1 - 1] - v;   // ids of N_H(v) lie in [v+1, v+window]
        const int mode = cta_mode(strategy, hv, window, work, smem_bytes);
        staged st{};
        st.hv = hv;
        st.h0 = h0;
        if (mode == MODE_BITMAP) {
            const int words = (int)((window + 31) >> 5);
            uint32_t* bits = (uint32_t*)dyn;
            uint32_t* rnk = bits + words;
            uint32_t* cnt = rnk + words;
            for (int i = threadIdx.x; i < words; i += nt) bits[i] = 0;
            for (int i = threadIdx.x; i < hv; i += nt) cnt[i] = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < hv; i += nt) {
                int32_t off = col[h0 + i] - base;
                atomicOr(&bits[off >> 5], 1u << (off & 31));
            }
            __syncthreads();
            // exclusive prefix of popcounts over the words: each thread owns a
            // contiguous slice, then a scan over the thread sums.
            const int per = (words + nt - 1) / nt;
            const int w0 = min(threadIdx.x * per, words), w1 = min(w0 + per, words);
            uint32_t sum = 0;
            for (int i = w0; i < w1; ++i) sum += __popc(bits[i]);
            uint32_t incl = sum;
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t x = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += x;
            }
            if (lane == 31) s_scan[warp] = incl;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t acc = 0;
                for (int k = 0; k < kCtaWarps; ++k) {
                    uint32_t x = s_scan[k];
                    s_scan[k] = acc;
                    acc += x;
                }
            }
            __syncthreads();
            uint32_t run = s_scan[warp] + incl - sum;
            for (int i = w0; i < w1; ++i) {
                rnk[i] = run;
                run += __popc(bits[i]);
            }
            __syncthreads();
            st.bits = bits;
            st.rank = rnk;
            st.cnt = cnt;
            st.base = base;
            st.nbits = (int32_t)window;
        } else if (mode == MODE_GLOBAL) {
            st.ids = col + h0;
        } else {
            int32_t* ids = (int32_t*)dyn;
            uint32_t* cnt = (uint32_t*)(ids + hv);
            for (int i = threadIdx.x; i < hv; i += nt) {
                ids[i] = col[h0 + i];
                cnt[i] = 0;
            }
            __syncthreads();
            st.ids = ids;
            st.cnt = cnt;
        }
        ull tv = 0;
        const int64_t first = pb + 32 * warp, stride = 32 * kCtaWarps;
        if (mode == MODE_BITMAP)
            run_batches<MODE_BITMAP>(lane, first, pe, stride, st, bsm[warp], col, twin, hrem, tri, flag, tv);
        else if (mode == MODE_MERGE)
            run_batches<MODE_MERGE>(lane, first, pe, stride, st, bsm[warp], col, twin, hrem, tri, flag, tv);
        else if (mode == MODE_GLOBAL)
            run_batches<MODE_GLOBAL>(lane, first, pe, stride, st, bsm[warp], col, twin, hrem, tri, flag, tv);
        else
            run_batches<MODE_BSEARCH>(lane, first, pe, stride, st, bsm[warp], col, twin, hrem, tri, flag, tv);
        tv = warp_sum(tv);
        if (lane == 0) s_tv[warp] = tv;
        __syncthreads();
        if (mode != MODE_GLOBAL) {
            for (int i = threadIdx.x; i < hv; i += nt) {
                uint32_t c = st.cnt[i];
                if (c) {
                    atomicAdd(&tri[col[h0 + i]], (ull)c);
                    flag[h0 + i] = 1;
                }
            }
        }
        if (threadIdx.x == 0) {
            ull t = 0;
            for (int k = 0; k < kCtaWarps; ++k) t += s_tv[k];
            if (t) {
                atomicAdd(&tri[v], t);
                atomicAdd(total, t);
            }
        }
    }
}

size_t g_cta_smem = 0;

tc_status ensure_cta_smem() {
    if (g_cta_smem) return TC_OK;
    int dev = 0, optin = 0;
    TC_CUDA(cudaGetDevice(&dev));
    TC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    size_t static_bytes = sizeof(batch_smem) * kCtaWarps + 256;
    size_t want = TC_CTA_SMEM;
    if ((size_t)optin < want + static_bytes) want = (size_t)optin - static_bytes;
    TC_CUDA(cudaFuncSetAttribute(k_count_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want));
    g_cta_smem = want;
    return TC_OK;
}

}  // namespace

tc_status run_count(tc_graph* g, cudaStream_t s) {
    const int64_t n = g->n, e2 = 2 * g->m;
    TC_CUDA(cudaMemsetAsync(g->tri, 0, (n + 1) * 8, s));
    TC_CUDA(cudaMemsetAsync(g->flag, 0, e2 + 16, s));
    TC_CUDA(cudaMemsetAsync(g->counters, 0, 8 * 8, s));
    ull* total = g->counters;
    const int sms = sm_count();
    if (g->plan.n_cta > 0 || (g->strategy == TC_STRATEGY_BITMAP && g->plan.n_warp > 0)) {
        TC_TRY(ensure_cta_smem());
    }
    // With the bitmap forced, warp items run through the CTA kernel too so
    // that every item uses (or falls back from) the bitmap.
    const bool warp_as_cta = g->strategy == TC_STRATEGY_BITMAP;
    if (g->plan.n_cta > 0) {
        launch_scope ls("count_cta", s);
        k_count_cta<<<sms * 1, TC_CTA_THREADS, g_cta_smem, s>>>(
            g->row_ptr, g->col, g->hstart, g->twin, g->hrem, g->plan.c_v, g->plan.c_pb,
            g->plan.c_pe, g->plan.n_cta, g->counters + 2, g->strategy, g_cta_smem, g->tri, g->flag,
            total);
        TC_LAUNCH_CHECK();
    }
    if (g->plan.n_warp > 0) {
        if (warp_as_cta) {
            launch_scope ls("count_cta", s);
            k_count_cta<<<sms * 1, TC_CTA_THREADS, g_cta_smem, s>>>(
                g->row_ptr, g->col, g->hstart, g->twin, g->hrem, g->plan.w_v, g->plan.w_pb,
                g->plan.w_pe, g->plan.n_warp, g->counters + 3, g->strategy, g_cta_smem, g->tri,
                g->flag, total);
            TC_LAUNCH_CHECK();
        } else {
            int per_sm = 0;
            TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_warp, TC_CTA_THREADS, 0));
            per_sm = std::max(per_sm, 1);
            launch_scope ls("count_warp", s);
            k_count_warp<<<sms * per_sm, TC_CTA_THREADS, 0, s>>>(
                g->row_ptr, g->col, g->hstart, g->twin, g->hrem, g->plan.w_v, g->plan.w_pb,
                g->plan.w_pe, g->plan.n_warp, g->counters + 1, g->strategy, g->tri, g->flag, total);
            TC_LAUNCH_CHECK();
        }
    }
    return TC_OK;
}

}  // namespace tcx
