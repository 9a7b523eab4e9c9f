// tc_count: triangle counts △(v), △(G) and edge flags (steps 1-2 of the
// elementary algorithm, section "Algorithm").
//
// Orientation as in Procedure 1: every triangle u < v < w (rank order) is
// met exactly once, from its middle vertex v and its lowest vertex u ∈ N_L(v),
// as an id w of N_H(u) that is also in N_H(v).  A work item is a middle
// vertex v with a range of its lower neighbours u.  The item stages N_H(v)
// on chip once (Procedure 1's marker array T: here a bitmap over the id
// window of N_H(v), or a sorted list) and streams, for every u of the item,
// only the part of N_H(u) above v — col[twin(u,v)+1 .. row_end(u)) — since
// ids at or below v cannot be in N_H(v).
//
// A hit (u, v, w) adds one to △(u), △(v), △(w), △(G) and marks the three
// edges.  Flags live on the canonical (tail) entry of each edge — the
// position of the higher end inside the lower end's N_H — the layout of the
// per-position arrays L_v of the appendix procedure ("Alternative Triangle
// Neighbor Algorithm"): (u,w) at the streamed position, (v,w) at the staged
// position, (u,v) at twin(u,v).
//
// Counts are aggregated on chip before the 64-bit integer atomics: per
// staged id (shared counters flushed once per item), per lower neighbour
// (one counter per batch segment), per middle vertex (a register).
//
// Streaming: a warp takes 32 lower neighbours at a time (a batch), keeps the
// non-empty streams as compacted segments and walks their concatenation
// with lane-consecutive ids (coalesced loads).  The segment of each lane is
// found from a 32-bit mask of the segment starts inside the current
// 32-id window (one warp OR-reduction), and every lane keeps 4 windows in
// flight.
#include <cub/cub.cuh>

#include <algorithm>

#include "tc_internal.cuh"

namespace tcx {

namespace {

typedef unsigned long long ull;

constexpr unsigned FULL = 0xffffffffu;
constexpr int kIlp = 4;                 // 32-id windows in flight per lane
constexpr int kCtaWarps = TC_CTA_THREADS / 32;

// Planner constants.
constexpr int64_t kBitmapSmallSmem = 44 * 1024;   // dynamic smem of the small-bitmap kernel
constexpr int64_t kBitmapLargeSmem = 180 * 1024;  // ... of the large-bitmap / CTA-list kernels
constexpr int64_t kCtaChunk = 65536;              // target wedges per CTA item
constexpr int64_t kWarpChunk = 32768;             // target wedges per warp item
constexpr int64_t kCtaMinWork = 4096;             // below this a vertex is a warp item

enum { L_BITMAP = 0, L_SORTED = 1, L_GLOBAL = 2 };

// ------------------------------------------------------------ lookups
// N_H(v) as a bitmap over [base, base + nbits): bit (w - base) set iff
// w ∈ N_H(v); rank[k] = set bits before word k gives w's staged index.
struct lookup_bitmap {
    const uint32_t* bits;
    const uint32_t* rank;
    int32_t base;
    int32_t nbits;
    __device__ __forceinline__ bool find(int32_t w, int& l) const {
        uint32_t off = (uint32_t)(w - base);
        if (off >= (uint32_t)nbits) return false;
        uint32_t word = bits[off >> 5];
        uint32_t bit = 1u << (off & 31);
        if (!(word & bit)) return false;
        l = (int)rank[off >> 5] + __popc(word & (bit - 1));
        return true;
    }
};

// N_H(v) as an ascending list in shared memory.
struct lookup_sorted {
    const int32_t* ids;
    int hv;
    __device__ __forceinline__ bool find(int32_t w, int& l) const {
        int lo = 0, len = hv;
        while (len > 0) {
            int half = len >> 1;
            if (ids[lo + half] < w) {
                lo += half + 1;
                len -= half + 1;
            } else {
                len = half;
            }
        }
        l = lo;
        return lo < hv && ids[lo] == w;
    }
};

// N_H(v) read in place from global memory (lists too long for shared memory).
struct lookup_global {
    const int32_t* ids;
    int hv;
    __device__ __forceinline__ bool find(int32_t w, int& l) const {
        int lo = 0, len = hv;
        while (len > 0) {
            int half = len >> 1;
            if (__ldg(ids + lo + half) < w) {
                lo += half + 1;
                len -= half + 1;
            } else {
                len = half;
            }
        }
        l = lo;
        return lo < hv && __ldg(ids + lo) == w;
    }
};

// ------------------------------------------------------------ batches
// The non-empty streams of one batch of 32 lower neighbours, compacted.
struct batch_smem {
    int64_t start[32];   // first streamed position: twin(u,v) + 1
    int32_t excl[32];    // offset of the stream in the batch's concatenation
    int32_t u[32];       // the lower neighbour
    uint32_t hits[32];   // triangles found on the stream
};

// Loads head entries [b, min(b+32, pe)); returns the concatenated length.
__device__ __forceinline__ int load_batch(int lane, int64_t b, int64_t pe,
                                          const int32_t* __restrict__ col,
                                          const int64_t* __restrict__ twin,
                                          const int32_t* __restrict__ hrem, batch_smem& bs,
                                          int& nseg, int& my_excl) {
    const int64_t p = b + lane;
    int r = 0;
    if (p < pe) r = hrem[p];
    int incl = r;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int x = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += x;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const unsigned nz = __ballot_sync(FULL, r > 0);
    if (r > 0) {
        const int k = __popc(nz & ((1u << lane) - 1));
        bs.start[k] = twin[p] + 1;
        bs.excl[k] = incl - r;
        bs.u[k] = col[p];
        bs.hits[k] = 0;
    }
    nseg = __popc(nz);
    __syncwarp();
    my_excl = lane < nseg ? bs.excl[lane] : 0x7fffffff;
    return total;
}

// Credits the hits of each stream to △(u) and flags the edge (u, v).
__device__ __forceinline__ void close_batch(int lane, int nseg, batch_smem& bs,
                                            ull* __restrict__ tri, uint8_t* __restrict__ flag,
                                            ull& tv) {
    __syncwarp();
    if (lane < nseg) {
        const uint32_t c = bs.hits[lane];
        if (c) {
            atomicAdd(&tri[bs.u[lane]], (ull)c);
            flag[bs.start[lane] - 1] = 1;   // twin(u, v): the canonical entry of (u, v)
            tv += c;
        }
    }
    __syncwarp();
}

// Walks the concatenated streams of a batch and looks every id up in the
// staged N_H(v).  CNT: per staged index counters in shared memory (else
// the counts of w go straight to global memory).
template <class LK, bool CNT>
__device__ __forceinline__ void stream_batch(int lane, int total, int my_excl, const LK& lk,
                                             batch_smem& bs, uint32_t* cnt, int64_t h0,
                                             const int32_t* __restrict__ col,
                                             ull* __restrict__ tri, uint8_t* __restrict__ flag) {
    const unsigned le = FULL >> (31 - lane);           // lanes 0..lane
    int s0 = -1;                                       // segment covering the id before the window
    for (int F = 0; F < total; F += 32 * kIlp) {
        int64_t pos[kIlp];
        int seg[kIlp];
        unsigned smask[kIlp];
        bool ok[kIlp];
        int32_t w[kIlp];
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const int Fk = F + 32 * k;
            const int rel = my_excl - Fk;
            const unsigned bit = (rel >= 0 && rel < 32) ? (1u << rel) : 0u;
            smask[k] = __reduce_or_sync(FULL, bit);
            seg[k] = s0 + __popc(smask[k] & le);
            s0 += __popc(smask[k]);
            const int f = Fk + lane;
            ok[k] = f < total;
            pos[k] = ok[k] ? bs.start[seg[k]] + (f - bs.excl[seg[k]]) : 0;
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) w[k] = ok[k] ? __ldg(col + pos[k]) : -1;
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            int l = 0;
            const bool hit = ok[k] && lk.find(w[k], l);
            const unsigned hm = __ballot_sync(FULL, hit);
            if (hm == 0) continue;
            if (hit) {
                if (CNT) {
                    atomicAdd(&cnt[l], 1u);
                } else {
                    atomicAdd(&tri[w[k]], 1ull);
                    flag[h0 + l] = 1;
                }
                flag[pos[k]] = 1;
            }
            // one shared atomic per (segment, window): the first lane of each
            // segment run adds the run's hits
            const bool leader = lane == 0 || ((smask[k] >> lane) & 1u);
            if (leader) {
                const unsigned above = smask[k] & ~le;
                const int end = above ? __ffs(above) - 1 : 32;
                const unsigned range = (end == 32 ? FULL : ((1u << end) - 1)) & ~((1u << lane) - 1);
                const unsigned c = __popc(hm & range);
                if (c) atomicAdd(&bs.hits[seg[k]], c);
            }
        }
    }
}

// Merge-path intersection of the staged A = N_H(v) (shared, ascending)
// with each stream B of the batch in turn.  The 32 lanes split the merge
// path of A and B into equal diagonals; on ties the A element is consumed
// first, and a common id is counted when its A element is consumed while
// the current B element equals it.
__device__ __forceinline__ void merge_batch(int lane, int nseg, const int32_t* A, int na,
                                            batch_smem& bs, uint32_t* cnt, int total,
                                            const int32_t* __restrict__ col,
                                            uint8_t* __restrict__ flag) {
    for (int s = 0; s < nseg; ++s) {
        const int nb = (s + 1 < nseg ? bs.excl[s + 1] : total) - bs.excl[s];
        const int32_t* B = col + bs.start[s];
        const int L = na + nb;
        const int d0 = (int)(((int64_t)L * lane) >> 5), d1 = (int)(((int64_t)L * (lane + 1)) >> 5);
        int lo = max(0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= __ldg(B + (d0 - mid - 1))) lo = mid + 1; else hi = mid;
        }
        int i = lo, j = d0 - lo;
        uint32_t found = 0;
        for (int d = d0; d < d1; ++d) {
            if (i < na && (j >= nb || A[i] <= __ldg(B + j))) {
                if (j < nb && __ldg(B + j) == A[i]) {
                    atomicAdd(&cnt[i], 1u);
                    flag[bs.start[s] + j] = 1;
                    ++found;
                }
                ++i;
            } else {
                ++j;
            }
        }
        for (int o = 16; o; o >>= 1) found += __shfl_xor_sync(FULL, found, o);
        if (lane == 0 && found) bs.hits[s] += found;
        __syncwarp();
    }
}

__device__ __forceinline__ ull warp_sum(ull x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// ------------------------------------------------------------ warp items
// One warp per item; N_H(v) (at most TC_WARP_CAP ids) staged as a sorted list.
struct warp_smem {
    int32_t ids[TC_WARP_CAP];
    uint32_t cnt[TC_WARP_CAP];
    batch_smem bs;
};

constexpr int kWarpItemsPerFetch = 4;

template <bool MERGE>
__global__ void __launch_bounds__(TC_CTA_THREADS)
k_count_warp(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
             const int64_t* __restrict__ hstart, const int64_t* __restrict__ twin,
             const int32_t* __restrict__ hrem, const int32_t* __restrict__ it_v,
             const int64_t* __restrict__ it_pb, const int64_t* __restrict__ it_pe,
             int64_t n_items, ull* __restrict__ cursor, ull* __restrict__ tri,
             uint8_t* __restrict__ flag, ull* __restrict__ total) {
    __shared__ warp_smem sm[kCtaWarps];
    const int lane = threadIdx.x & 31;
    warp_smem& ws = sm[threadIdx.x >> 5];
    ull tv_all = 0;
    for (;;) {
        int64_t base = 0;
        if (lane == 0) base = (int64_t)atomicAdd(cursor, (ull)kWarpItemsPerFetch);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n_items) break;
        const int64_t lim = min(base + kWarpItemsPerFetch, n_items);
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
            const lookup_sorted lk{ws.ids, hv};
            ull tv = 0;
            for (int64_t b = pb; b < pe; b += 32) {
                int nseg, my_excl;
                const int tot = load_batch(lane, b, pe, col, twin, hrem, ws.bs, nseg, my_excl);
                if (tot > 0) {
                    if (MERGE) merge_batch(lane, nseg, ws.ids, hv, ws.bs, ws.cnt, tot, col, flag);
                    else stream_batch<lookup_sorted, true>(lane, tot, my_excl, lk, ws.bs, ws.cnt, h0, col, tri, flag);
                }
                close_batch(lane, nseg, ws.bs, tri, flag, tv);
            }
            __syncwarp();
            for (int i = lane; i < hv; i += 32) {
                const uint32_t c = ws.cnt[i];
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
// One CTA per item; the 8 warps share the staged N_H(v) and take the
// item's batches round-robin.
template <int LOOK, bool MERGE>
__global__ void __launch_bounds__(TC_CTA_THREADS)
k_count_cta(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
            const int64_t* __restrict__ hstart, const int64_t* __restrict__ twin,
            const int32_t* __restrict__ hrem, const int32_t* __restrict__ it_v,
            const int64_t* __restrict__ it_pb, const int64_t* __restrict__ it_pe,
            int64_t n_items, ull* __restrict__ cursor, ull* __restrict__ tri,
            uint8_t* __restrict__ flag, ull* __restrict__ total) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ batch_smem bsm[kCtaWarps];
    __shared__ int64_t s_item;
    __shared__ ull s_tv[kCtaWarps];
    __shared__ uint32_t s_scan[kCtaWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = TC_CTA_THREADS;
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
        uint32_t* cnt = nullptr;
        lookup_bitmap lb{};
        lookup_sorted ls{};
        lookup_global lg{};
        if (LOOK == L_BITMAP) {
            // ids of N_H(v) lie in [v+1, col[h1-1]]
            const int32_t base = v + 1;
            const int32_t nbits = col[h1 - 1] - v;
            const int words = (nbits + 31) >> 5;
            uint32_t* bits = (uint32_t*)dyn;
            uint32_t* rnk = bits + words;
            cnt = rnk + words;
            for (int i = threadIdx.x; i < words; i += nt) bits[i] = 0;
            for (int i = threadIdx.x; i < hv; i += nt) cnt[i] = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < hv; i += nt) {
                const int32_t off = col[h0 + i] - base;
                atomicOr(&bits[off >> 5], 1u << (off & 31));
            }
            __syncthreads();
            // rank[k] = set bits in words [0, k): per-thread slices, warp
            // scan of the slice sums, then a scan over the 8 warp totals
            const int per = (words + nt - 1) / nt;
            const int w0 = min((int)threadIdx.x * per, words), w1 = min(w0 + per, words);
            uint32_t sum = 0;
            for (int i = w0; i < w1; ++i) sum += __popc(bits[i]);
            uint32_t incl = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t x = __shfl_up_sync(FULL, incl, d);
                if (lane >= d) incl += x;
            }
            if (lane == 31) s_scan[warp] = incl;
            __syncthreads();
            uint32_t before = 0;
            for (int k = 0; k < warp; ++k) before += s_scan[k];
            uint32_t run = before + incl - sum;
            for (int i = w0; i < w1; ++i) {
                rnk[i] = run;
                run += __popc(bits[i]);
            }
            __syncthreads();
            lb = lookup_bitmap{bits, rnk, base, nbits};
        } else if (LOOK == L_SORTED) {
            int32_t* ids = (int32_t*)dyn;
            cnt = (uint32_t*)(ids + hv);
            for (int i = threadIdx.x; i < hv; i += nt) {
                ids[i] = col[h0 + i];
                cnt[i] = 0;
            }
            __syncthreads();
            ls = lookup_sorted{ids, hv};
        } else {
            lg = lookup_global{col + h0, hv};
        }
        ull tv = 0;
        batch_smem& bs = bsm[warp];
        for (int64_t b = pb + 32 * warp; b < pe; b += 32 * kCtaWarps) {
            int nseg, my_excl;
            const int tot = load_batch(lane, b, pe, col, twin, hrem, bs, nseg, my_excl);
            if (tot > 0) {
                if (LOOK == L_BITMAP)
                    stream_batch<lookup_bitmap, true>(lane, tot, my_excl, lb, bs, cnt, h0, col, tri, flag);
                else if (LOOK == L_SORTED && MERGE)
                    merge_batch(lane, nseg, ls.ids, hv, bs, cnt, tot, col, flag);
                else if (LOOK == L_SORTED)
                    stream_batch<lookup_sorted, true>(lane, tot, my_excl, ls, bs, cnt, h0, col, tri, flag);
                else
                    stream_batch<lookup_global, false>(lane, tot, my_excl, lg, bs, nullptr, h0, col, tri, flag);
            }
            close_batch(lane, nseg, bs, tri, flag, tv);
        }
        tv = warp_sum(tv);
        if (lane == 0) s_tv[warp] = tv;
        __syncthreads();
        if (LOOK != L_GLOBAL) {
            for (int i = threadIdx.x; i < hv; i += nt) {
                const uint32_t c = cnt[i];
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

// ------------------------------------------------------------ planner
struct class_acc {
    unsigned long long items[TC_NUM_CLS];
    unsigned long long staged[TC_NUM_CLS];
    unsigned long long head[TC_NUM_CLS];
    unsigned long long wedges[TC_NUM_CLS];
};

// Class and chunk count of every middle vertex; rows visited in reverse
// rank order so that the heaviest vertices come first in every class.
__global__ void k_classify(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                           const int32_t* __restrict__ col, const int64_t* __restrict__ work,
                           int64_t n, int strategy, int64_t* __restrict__ cnt,
                           int8_t* __restrict__ cls, class_acc* __restrict__ acc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = n - 1 - i;
        const int64_t b = row_ptr[r], h = hstart[r], e = row_ptr[r + 1];
        const int64_t hv = e - h, lv = h - b, W = work[r];
        int c = -1;
        int64_t chunks = 0;
        if (W > 0 && hv > 0) {
            const int64_t nbits = (int64_t)col[e - 1] - r;
            const int64_t words = (nbits + 31) >> 5;
            const int64_t bm_bytes = 8 * words + 4 * hv;
            const bool fit_s = bm_bytes <= kBitmapSmallSmem;
            const bool fit_l = bm_bytes <= kBitmapLargeSmem;
            const bool bitmap_ok = strategy == TC_STRATEGY_BITMAP ||
                                   (strategy == TC_STRATEGY_AUTO && W >= kCtaMinWork && W >= 2 * words);
            if (strategy == TC_STRATEGY_GLOBAL) c = TC_CLS_CTA_LIST;
            else if (bitmap_ok && fit_s) c = TC_CLS_BITMAP_S;
            else if (bitmap_ok && fit_l) c = TC_CLS_BITMAP_L;
            else if (hv <= TC_WARP_CAP) c = TC_CLS_WARP;
            else c = TC_CLS_CTA_LIST;
            const int64_t chunk = c == TC_CLS_WARP ? kWarpChunk : kCtaChunk;
            chunks = (W + chunk - 1) / chunk;
            if (chunks > lv) chunks = lv;
            if (chunks < 1) chunks = 1;
            atomicAdd(&acc->items[c], (ull)chunks);
            atomicAdd(&acc->staged[c], (ull)hv);
            atomicAdd(&acc->head[c], (ull)lv);
            atomicAdd(&acc->wedges[c], (ull)W);
        }
        cls[i] = (int8_t)c;
        for (int k = 0; k < TC_NUM_CLS; ++k) cnt[k * (n + 1) + i] = (k == c) ? chunks : 0;
    }
}

__global__ void k_emit(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                       int64_t n, const int8_t* __restrict__ cls, const int64_t* __restrict__ cnt,
                       const int64_t* __restrict__ off, int32_t* v0, int64_t* pb0, int64_t* pe0,
                       int32_t* v1, int64_t* pb1, int64_t* pe1, int32_t* v2, int64_t* pb2,
                       int64_t* pe2, int32_t* v3, int64_t* pb3, int64_t* pe3) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cls[i];
        if (c < 0) continue;
        const int64_t r = n - 1 - i;
        const int64_t b = row_ptr[r], lv = hstart[r] - b;
        const int64_t k = cnt[c * (n + 1) + i], o = off[c * (n + 1) + i];
        int32_t* vv = c == 0 ? v0 : c == 1 ? v1 : c == 2 ? v2 : v3;
        int64_t* pbb = c == 0 ? pb0 : c == 1 ? pb1 : c == 2 ? pb2 : pb3;
        int64_t* pee = c == 0 ? pe0 : c == 1 ? pe1 : c == 2 ? pe2 : pe3;
        for (int64_t j = 0; j < k; ++j) {
            vv[o + j] = (int32_t)r;
            pbb[o + j] = b + lv * j / k;
            pee[o + j] = b + lv * (j + 1) / k;
        }
    }
}

inline int blocks_for(int64_t items) {
    int64_t b = (items + 255) / 256, cap = (int64_t)sm_count() * 16;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

template <class K>
tc_status launch_persistent(K kernel, const char* name, size_t smem, int64_t items, cudaStream_t s,
                            const tc_graph* g, const tc_plan& p, int c, ull* cursor) {
    if (items == 0) return TC_OK;
    // static + dynamic shared memory may exceed the 48 KB default
    if (smem > 0) TC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, TC_CTA_THREADS, smem));
    per_sm = std::max(per_sm, 1);
    int64_t blocks = std::min<int64_t>((int64_t)sm_count() * per_sm, items);
    launch_scope ls(name, s);
    kernel<<<(int)blocks, TC_CTA_THREADS, smem, s>>>(g->row_ptr, g->col, g->hstart, g->twin, g->hrem,
                                                     p.v[c], p.pb[c], p.pe[c], items, cursor, g->tri,
                                                     g->flag, g->counters);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

void free_plan(tc_plan& p, cudaStream_t s) {
    for (int c = 0; c < TC_NUM_CLS; ++c) {
        dfree(p.v[c], s);
        dfree(p.pb[c], s);
        dfree(p.pe[c], s);
        p.v[c] = nullptr;
        p.pb[c] = p.pe[c] = nullptr;
        p.count[c] = 0;
    }
    p.strategy = -1;
}

tc_status make_plan(tc_graph* g, int strategy, cudaStream_t s) {
    free_plan(g->plan, s);
    tc_plan& p = g->plan;
    const int64_t n = g->n;
    int64_t* cnt = nullptr;
    int64_t* off = nullptr;
    int8_t* cls = nullptr;
    class_acc* acc = nullptr;
    uint8_t* tmp = nullptr;
    size_t tmp_bytes = 0;
    tc_status st = TC_OK;
    auto cleanup = [&]() {
        dfree(cnt, s);
        dfree(off, s);
        dfree(cls, s);
        dfree(acc, s);
        dfree(tmp, s);
    };
#define PLAN_TRY(x)              \
    do {                         \
        st = (x);                \
        if (st < 0) {            \
            cleanup();           \
            return st;           \
        }                        \
    } while (0)
#define PLAN_CUDA(x) PLAN_TRY(from_cuda(x))
    PLAN_TRY(dalloc((void**)&cnt, TC_NUM_CLS * (n + 1) * 8, s));
    PLAN_TRY(dalloc((void**)&off, TC_NUM_CLS * (n + 1) * 8, s));
    PLAN_TRY(dalloc((void**)&cls, n + 1, s));
    PLAN_TRY(dalloc((void**)&acc, sizeof(class_acc), s));
    PLAN_CUDA(cudaMemsetAsync(acc, 0, sizeof(class_acc), s));
    PLAN_CUDA(cudaMemsetAsync(cnt, 0, TC_NUM_CLS * (n + 1) * 8, s));
    if (n > 0) {
        launch_scope ls("plan_classify", s);
        k_classify<<<blocks_for(n), 256, 0, s>>>(g->row_ptr, g->hstart, g->col, g->work, n, strategy,
                                                  cnt, cls, acc);
        PLAN_CUDA(cudaGetLastError());
    }
    PLAN_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, cnt, off, n + 1, s));
    PLAN_TRY(dalloc((void**)&tmp, tmp_bytes, s));
    {
        launch_scope ls("plan_scan", s);
        for (int c = 0; c < TC_NUM_CLS; ++c)
            PLAN_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt + c * (n + 1), off + c * (n + 1),
                                                    n + 1, s));
    }
    class_acc h{};
    PLAN_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    PLAN_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < TC_NUM_CLS; ++c) {
        p.count[c] = (int64_t)h.items[c];
        PLAN_TRY(dalloc((void**)&p.v[c], (p.count[c] + 1) * 4, s));
        PLAN_TRY(dalloc((void**)&p.pb[c], (p.count[c] + 1) * 8, s));
        PLAN_TRY(dalloc((void**)&p.pe[c], (p.count[c] + 1) * 8, s));
    }
    if (n > 0) {
        launch_scope ls("plan_emit", s);
        k_emit<<<blocks_for(n), 256, 0, s>>>(g->row_ptr, g->hstart, n, cls, cnt, off, p.v[0], p.pb[0],
                                             p.pe[0], p.v[1], p.pb[1], p.pe[1], p.v[2], p.pb[2],
                                             p.pe[2], p.v[3], p.pb[3], p.pe[3]);
        PLAN_CUDA(cudaGetLastError());
    }
    p.smem[TC_CLS_BITMAP_S] = kBitmapSmallSmem;
    p.smem[TC_CLS_BITMAP_L] = kBitmapLargeSmem;
    p.smem[TC_CLS_WARP] = 0;
    p.smem[TC_CLS_CTA_LIST] = kBitmapLargeSmem;
    p.strategy = strategy;
    // algorithmic bytes of each class's kernel: stage N_H(v) once (4 hv),
    // read each head entry's label, twin and stream length (16), stream each
    // wedge id (4)
    tc_graph_stats& S = g->stats;
    for (int c = 0; c < TC_NUM_CLS; ++c) {
        S.items[c] = p.count[c];
        S.class_bytes[c] = 4.0 * (double)h.staged[c] + 16.0 * (double)h.head[c] + 4.0 * (double)h.wedges[c];
    }
    cleanup();
    PLAN_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
#undef PLAN_TRY
#undef PLAN_CUDA
}

tc_status run_count(tc_graph* g, cudaStream_t s) {
    const int64_t n = g->n, e2 = 2 * g->m;
    if (g->plan.strategy != g->strategy) TC_TRY(make_plan(g, g->strategy, s));
    TC_CUDA(cudaMemsetAsync(g->tri, 0, (n + 1) * 8, s));
    TC_CUDA(cudaMemsetAsync(g->flag, 0, e2 + 16, s));
    TC_CUDA(cudaMemsetAsync(g->counters, 0, 8 * 8, s));
    const tc_plan& p = g->plan;
    ull* cur = g->counters + 1;
    const bool merge = g->strategy == TC_STRATEGY_MERGE;
    // heaviest classes first; each kernel drains its own item queue
    TC_TRY(launch_persistent(k_count_cta<L_BITMAP, false>, "count_bitmap_l", p.smem[TC_CLS_BITMAP_L],
                             p.count[TC_CLS_BITMAP_L], s, g, p, TC_CLS_BITMAP_L, cur + TC_CLS_BITMAP_L));
    TC_TRY(launch_persistent(k_count_cta<L_BITMAP, false>, "count_bitmap_s", p.smem[TC_CLS_BITMAP_S],
                             p.count[TC_CLS_BITMAP_S], s, g, p, TC_CLS_BITMAP_S, cur + TC_CLS_BITMAP_S));
    if (p.count[TC_CLS_CTA_LIST] > 0) {
        // lists longer than the shared budget are searched in place
        const bool fits = g->strategy != TC_STRATEGY_GLOBAL &&
                          (int64_t)g->stats.max_out_degree * 8 <= (int64_t)p.smem[TC_CLS_CTA_LIST];
        if (fits && merge)
            TC_TRY(launch_persistent(k_count_cta<L_SORTED, true>, "count_cta_list", p.smem[TC_CLS_CTA_LIST],
                                     p.count[TC_CLS_CTA_LIST], s, g, p, TC_CLS_CTA_LIST, cur + TC_CLS_CTA_LIST));
        else if (fits)
            TC_TRY(launch_persistent(k_count_cta<L_SORTED, false>, "count_cta_list", p.smem[TC_CLS_CTA_LIST],
                                     p.count[TC_CLS_CTA_LIST], s, g, p, TC_CLS_CTA_LIST, cur + TC_CLS_CTA_LIST));
        else
            TC_TRY(launch_persistent(k_count_cta<L_GLOBAL, false>, "count_cta_global", 0,
                                     p.count[TC_CLS_CTA_LIST], s, g, p, TC_CLS_CTA_LIST, cur + TC_CLS_CTA_LIST));
    }
    if (merge)
        TC_TRY(launch_persistent(k_count_warp<true>, "count_warp", 0, p.count[TC_CLS_WARP], s, g, p,
                                 TC_CLS_WARP, cur + TC_CLS_WARP));
    else
        TC_TRY(launch_persistent(k_count_warp<false>, "count_warp", 0, p.count[TC_CLS_WARP], s, g, p,
                                 TC_CLS_WARP, cur + TC_CLS_WARP));
    return TC_OK;
}

}  // namespace tcx
