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
// (one counter per stream), per middle vertex (a register).
//
// Streaming: a batch of head entries (32 for a warp item, 256 per round for
// a CTA item) becomes a compacted table of streams, read in 8-aligned
// octets of ids — one 32-byte load, a whole sector, per octet — with ids
// outside the stream masked; each lane takes G consecutive octets per
// window and finds its stream from a 32-bit mask of the stream starts in
// the window (one warp OR-reduction).
//
// Item classes (planner below): CTA bitmaps of two shared sizes, warp
// items (bitmap, or sorted list behind a hashed filter), CTA sorted lists
// (shared or global), and
// one thread per tiny vertex.  Two switches ride along every kernel: the
// edge-count mode (EC), which adds per-entry triangle counts where the
// normal mode sets flag bits, and an item offset/stride, which restricts a
// launch to one shard's share of the items.
#include <cub/cub.cuh>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "tc_internal.cuh"

namespace tcx {

namespace {

typedef unsigned long long ull;

constexpr unsigned FULL = 0xffffffffu;
constexpr int kCtaWarps = TC_CTA_THREADS / 32;
// threads of the CTA-item kernel (one head entry per thread per round)
#ifndef TC_CTA_ITEM_THREADS
#define TC_CTA_ITEM_THREADS 256
#endif
constexpr int kCtaT = TC_CTA_ITEM_THREADS;
constexpr int kCtaItemWarps = kCtaT / 32;
// CTA chunk target below which the small-bitmap class runs 2 kCtaT threads
#ifndef TC_WIDE_CTA_CHUNK
#define TC_WIDE_CTA_CHUNK (1 << 17)
#endif
constexpr int64_t kWideCtaChunk = TC_WIDE_CTA_CHUNK;
// The large-bitmap class (100 KB of shared memory, two CTAs per SM) runs
// 16-warp CTAs, so that an SM holds 32 warps instead of 16 (R-MAT scale
// 24: 2.22 -> 2.14 ms)
#ifndef TC_WIDE_L
#define TC_WIDE_L 1
#endif
#ifndef TC_CTA_MIN_BLOCKS
#define TC_CTA_MIN_BLOCKS (1024 / TC_CTA_ITEM_THREADS)   // CTAs per SM the CTA-item kernels are compiled for
#endif

// Planner constants.
// 40 KB keeps four CTAs per SM (the register limit) with room left for L1
#ifndef TC_BM_S_KB
#define TC_BM_S_KB 40
#endif
constexpr int64_t kBitmapSmallSmem = TC_BM_S_KB * 1024;   // dynamic smem of the small-bitmap CTA kernel
#ifndef TC_TIGHT_SMEM
#define TC_TIGHT_SMEM 1   // bitmap kernels sized to their largest item (below)
#endif
#ifndef TC_BM_L_KB
#define TC_BM_L_KB 100
#endif
constexpr int64_t kBitmapLargeSmem = TC_BM_L_KB * 1024;  // ... of the large-bitmap CTA kernel
constexpr int64_t kCtaListSmem = 100 * 1024;      // ... of the CTA sorted-list kernel

enum { L_BITMAP = 0, L_SORTED = 1, L_GLOBAL = 2 };

// ------------------------------------------------------------ lookups
// N_H(v) as a bitmap over the id window [base, base + nbits), base = v + 1,
// in 32-bit entries of 16 ids each: the low half holds the membership bits
// of ids [16 i, 16 i + 16) of the window, the high half the number of
// members before them (16 bits suffice since |N_H(v)| <= sqrt(2m) < 2^16).
// One shared load answers both "is w in N_H(v)" and "at which staged index".
// The offset nbits is never a member (the entry after the window is a zero
// guard), so an id outside the window is clamped onto it and the test
// needs no branch.
struct lookup_bitmap {
    const uint32_t* bits;   // the entries
    int32_t base;
    int32_t nbits;
    int32_t hv;             // staged ids (counters)
    __device__ __forceinline__ bool find(int32_t w, int& l) const {
        const uint32_t off = min((uint32_t)(w - base), (uint32_t)nbits);
        const uint32_t e = bits[TC_IX(off >> 4, (nbits >> 4) + 1)];
        if (!((e >> (off & 15)) & 1u)) return false;
        l = (int)(e >> 16) + __popc(e & ((1u << (off & 15)) - 1));
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
            const int half = len >> 1;
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

// N_H(v) as an ascending list behind a hashed filter: one bit per slot of a
// table of kFilterBits slots, set for the slot of every staged id.  An id
// whose slot is clear is not staged, which one shared load settles; only
// the others are bisected.  Light middle vertices (the warp items) have
// id windows far too wide for a bitmap, and almost every streamed id
// misses their N_H(v) (2 % hits at R-MAT scale 20), so the filter takes
// the bisection off nearly every id.
#ifndef TC_FILTER_LOG2
#define TC_FILTER_LOG2 13
#endif
constexpr int kFilterBits = 1 << TC_FILTER_LOG2;
constexpr int kFilterWords = kFilterBits / 32;
#ifndef TC_FILTER_HASHES
#define TC_FILTER_HASHES 2
#endif
// Fibonacci hashing: the top bits of the id times 2^32 / golden ratio (a
// second slot, with TC_FILTER_HASHES 2, from another odd multiplier)
__device__ __forceinline__ uint32_t filter_slot(int32_t w) {
    return ((uint32_t)w * 0x9E3779B1u) >> (32 - TC_FILTER_LOG2);
}
__device__ __forceinline__ uint32_t filter_slot2(int32_t w) {
    return ((uint32_t)w * 0x85EBCA6Bu) >> (32 - TC_FILTER_LOG2);
}
struct lookup_filtered {
    lookup_sorted ls;
    const uint32_t* filt;
};

// N_H(v) read in place from global memory (lists too long for shared memory).
struct lookup_global {
    const int32_t* ids;
    int hv;
    __device__ __forceinline__ bool find(int32_t w, int& l) const {
        int lo = 0, len = hv;
        while (len > 0) {
            const int half = len >> 1;
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

// Shared bytes of a bitmap staging: 16-id entries (+ guard, padded to even)
// and per-id counters; `words` is the window in 32-id units.
__host__ __device__ __forceinline__ int64_t bitmap_bytes(int64_t words, int64_t hv) {
    return 4 * (2 * words + 2) + 4 * hv;
}

__device__ __forceinline__ ull warp_sum(ull x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Builds a bitmap staging with threads t of nt; barrier() separates phases.
template <class Barrier>
__device__ __forceinline__ lookup_bitmap build_bitmap(int t, int nt, uint8_t* region, int32_t v,
                                                      int64_t h0, int hv, int32_t nbits,
                                                      const int32_t* __restrict__ col,
                                                      uint32_t*& cnt, Barrier barrier,
                                                      uint32_t* scan_tmp, int lane, int warp, int nwarps,
                                                      const tc_dims& dm) {
    // entry i: membership bits of ids [16 i, 16 i + 16) of the window in its
    // low half, the members before it in its high half
    const int ents = (nbits + 15) >> 4;
    uint32_t* ent = (uint32_t*)region;                      // ents + 1 (guard)
    cnt = ent + ((ents + 2) & ~1);
    const int32_t base = v + 1;
    for (int i = t; i <= ents; i += nt) ent[i] = 0;
    for (int i = t; i < hv; i += nt) cnt[i] = 0;
    barrier();
    for (int i = t; i < hv; i += nt) {
        const int32_t off = col[TC_IX(h0 + i, dm.e2 + 32)] - base;
        atomicOr(&ent[TC_IX(off >> 4, ents + 1)], 1u << (off & 15));
    }
    barrier();
    const int per = (ents + nt - 1) / nt;
    const int e0 = min(t * per, ents), e1 = min(e0 + per, ents);
    uint32_t sum = 0;
    for (int i = e0; i < e1; ++i) sum += __popc(ent[i]);
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t x = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += x;
    }
    uint32_t before = 0;
    if (nwarps > 1) {
        if (lane == 31) scan_tmp[warp] = incl;
        barrier();
        for (int k = 0; k < warp; ++k) before += scan_tmp[k];
    }
    uint32_t run = before + incl - sum;
    for (int i = e0; i < e1; ++i) {
        const uint32_t x = ent[i];
        ent[i] = x | (run << 16);
        run += __popc(x);
    }
    barrier();
    return lookup_bitmap{ent, base, nbits, hv};
}

// ------------------------------------------------------------ streams
// A batch of head entries (lower neighbours u of the item's middle vertex
// v) gives one stream per non-empty entry: col[p0, p0 + len), the part of
// N_H(u) above v (p0 = twin(u,v) + 1).  A stream is read in octets: 8 ids
// at an 8-aligned position, one 32-byte load (one whole sector), starting
// at p0 & ~7; a lane takes G consecutive octets per window, and ids outside
// [p0, p0 + len) are masked.  The table holds the batch's non-empty
// streams, compacted.
template <int N>
struct stream_table {
    int64_t va[N];        // first octet of the stream (8-aligned position)
    int32_t fl[N];        // (len << 3) | (p0 - va)
    int32_t u[N];
    uint32_t hits[N];
    int32_t gpre[N + 1];  // groups of G octets before each stream
};

// A head entry as loaded from global memory.
struct entry {
    int r;         // stream length hrem
    int32_t u;     // the lower neighbour
    int64_t t;     // twin(u, v)
};

__device__ __forceinline__ entry fetch_entry(int64_t p, int64_t pe, const tc_head* __restrict__ head,
                                             const tc_dims& dm) {
    entry e{0, 0, 0};
    if (p < pe) {
        const tc_head rec = head[TC_IX(p, dm.e2)];   // one 16-byte load
        e.r = rec.hrem;
        e.t = rec.twin;
        e.u = rec.u;
    }
    return e;
}

// Number of G-octet groups of an entry's stream (0 if empty).
template <int G>
__device__ __forceinline__ int entry_groups(const entry& e) {
    if (e.r == 0) return 0;
    const int64_t p0 = e.t + 1;
    const int octets = (int)((((p0 + e.r + 7) & ~7ll) - (p0 & ~7ll)) >> 3);
    return (octets + G - 1) / G;
}

template <int N>
__device__ __forceinline__ void put_stream(const entry& e, int k, int gpre, stream_table<N>& tb) {
    const int64_t p0 = e.t + 1;
    const int64_t va = p0 & ~7ll;
    tb.va[k] = va;
    tb.fl[k] = (e.r << 3) | (int)(p0 - va);
    tb.u[k] = e.u;
    tb.hits[k] = 0;
    tb.gpre[k] = gpre;
}

// Marks edge entries that lie in triangles.  Normally `f` holds one flag
// bit per CSR position; in edge-count mode (EC) it holds one 32-bit
// counter per CSR position and a mark adds the number of triangles found
// on that entry, giving t(u, v) = (A² ∘ A)(u, v) on every canonical entry.
template <bool EC>
__device__ __forceinline__ void mark(uint32_t* __restrict__ f, int64_t p, uint32_t c, const tc_dims& dm) {
    if (EC) atomicAdd(&f[TC_IX(p, dm.e2 + 1)], c);
    else flag_set(f, TC_IX(p, dm.fw * 32));
}
// The hits hm (bit k: position pos + k) of one octet (pos 8-aligned).
template <bool EC>
__device__ __forceinline__ void mark_octet(uint32_t* __restrict__ f, int64_t pos, uint32_t hm, const tc_dims& dm) {
    if (EC) {
        while (hm) {
            const int k = __ffs(hm) - 1;
            hm &= hm - 1;
            atomicAdd(&f[TC_IX(pos + k, dm.e2 + 1)], 1u);
        }
    } else if (hm) {
        // the octet's 8 flag bits lie in one 32-bit word
        flag_or(f, TC_IX(pos >> 5, dm.fw), hm << (pos & 31));
    }
}

// Credits the hits of stream k to △(u) and flags the edge (u, v).
template <int N, bool EC>
__device__ __forceinline__ void close_stream(int k, stream_table<N>& tb, ull* __restrict__ tri,
                                             uint32_t* __restrict__ flag, ull& tv, const tc_dims& dm) {
    const uint32_t c = tb.hits[k];
    if (c) {
        atomicAdd(&tri[TC_IX(tb.u[k], dm.n)], (ull)c);
        mark<EC>(flag, tb.va[k] + (tb.fl[k] & 7) - 1, c, dm);   // twin(u, v): the canonical entry of (u, v)
        tv += c;
    }
}

// 8 ids from an 8-aligned position: one 256-bit read-only load.
struct octet {
    int32_t x[8];
};
__device__ __forceinline__ octet load8(const int32_t* __restrict__ col, int64_t pos) {
    octet o;
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(o.x[0]), "=r"(o.x[1]), "=r"(o.x[2]), "=r"(o.x[3]), "=r"(o.x[4]), "=r"(o.x[5]),
                   "=r"(o.x[6]), "=r"(o.x[7])
                 : "l"(col + pos));
    return o;
}

// One octet (8 ids at the 8-aligned position pos, the first at offset off
// from the stream start): ids with offset in [0, len) are looked up; a hit
// counts the triangle (u, v, w) at the staged index, and the octet's hit
// flags are set with one 32-bit OR (its 8 flag bits lie in one word, and an
// OR never clears a flag another thread set).  Returns the hits.
template <class LK, bool CNT, bool EC>
__device__ __forceinline__ uint32_t visit_octet(const LK& lk, const octet& o, int64_t pos, int off, int len,
                                                uint32_t* cnt, int64_t h0, ull* __restrict__ tri,
                                                uint32_t* __restrict__ flag, const tc_dims& dm) {
    uint32_t bits = 0;
    uint32_t nh = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int l = 0;
        if ((unsigned)(off + k) < (unsigned)len && lk.find(o.x[k], l)) {
            if (CNT) {
                atomicAdd(&cnt[TC_IX(l, lk.hv)], 1u);
            } else {
                atomicAdd(&tri[TC_IX(o.x[k], dm.n)], 1ull);
                mark<EC>(flag, h0 + l, 1u, dm);
            }
            bits |= 1u << k;
            ++nh;
        }
    }
    mark_octet<EC>(flag, pos, bits, dm);
    return nh;
}

// The bitmap form in explicit phases — the 8 entry loads, the hit mask, the
// staged indices of the hits, then the counter atomics — so that the loads
// of an octet overlap instead of each waiting behind the previous id's
// atomic.
#ifndef TC_OCTET_ROTATE
#define TC_OCTET_ROTATE 1
#endif
// Ids of an octet inside its stream: bits [max(0, -off), min(8, len - off)).
__device__ __forceinline__ uint32_t octet_valid(int off, int len) {
    const int lo = off < 0 ? -off : 0;
    const int hi = len - off < 8 ? len - off : 8;
    return hi > lo ? (0xffu >> (8 - hi)) & (0xffu << lo) : 0u;
}

// The hit mask of one octet against a bitmap staging, with the hits counted
// at their staged indices; the caller sets the octet's flags.
// Staged index of the id at offset boff of a bitmap entry: the members
// before the entry plus those below bit s = boff & 15 in it (bits [0, s)
// shifted to the top by a clamped funnel shift, which gives 0 for s = 0).
__device__ __forceinline__ int staged_index(uint32_t word, uint32_t boff) {
    return (int)(word >> 16) + __popc(__funnelshift_lc(0u, word, 32u - (boff & 15u)));
}

// Ids of G consecutive octets inside their stream, bit 8 j + k for id k of
// octet j: bits [max(0, -off), min(8 G, len - off)).
template <int G>
__device__ __forceinline__ uint32_t group_valid(int off, int len) {
    static_assert(8 * G <= 32, "one 32-bit mask per group");
    const int lo = off < 0 ? -off : 0;
    const int hi = len - off < 8 * G ? len - off : 8 * G;
    const uint32_t full = 8 * G == 32 ? 0xffffffffu : (1u << (8 * G)) - 1;
    return hi > lo ? (full >> (8 * G - hi)) & (full << lo) : 0u;
}

// The hit mask of one octet against a bitmap staging (valid: the octet's
// ids inside the stream), hits counted at their staged indices.
__device__ __forceinline__ uint32_t octet_hits_masked(const lookup_bitmap& lk, const octet& o, uint32_t valid,
                                                      uint32_t* cnt) {
    uint32_t word[8], boff[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        boff[k] = min((uint32_t)(o.x[k] - lk.base), (uint32_t)lk.nbits);
        word[k] = lk.bits[TC_IX(boff[k] >> 4, (lk.nbits >> 4) + 1)];
    }
    uint32_t hm = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        hm |= __funnelshift_l(word[k], word[k], (uint32_t)k - (boff[k] & 15u)) & (1u << k);
    hm &= valid;
    int l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        l[k] = staged_index(word[k], boff[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if ((hm >> k) & 1u) atomicAdd(&cnt[TC_IX(l[k], lk.hv)], 1u);
    return hm;
}

__device__ __forceinline__ uint32_t octet_hits_bitmap(const lookup_bitmap& lk, const octet& o, int off, int len,
                                                      uint32_t* cnt) {
    uint32_t word[8], boff[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        boff[k] = min((uint32_t)(o.x[k] - lk.base), (uint32_t)lk.nbits);
        word[k] = lk.bits[TC_IX(boff[k] >> 4, (lk.nbits >> 4) + 1)];
    }
    uint32_t hm = 0;
    if (TC_OCTET_ROTATE) {
        // membership bit s = boff & 15 of each entry rotated onto bit k, then
        // the octet's ids outside the stream masked once
#pragma unroll
        for (int k = 0; k < 8; ++k)
            hm |= __funnelshift_l(word[k], word[k], (uint32_t)k - (boff[k] & 15u)) & (1u << k);
        hm &= octet_valid(off, len);
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            hm |= (((word[k] >> (boff[k] & 15)) & 1u) & ((unsigned)(off + k) < (unsigned)len ? 1u : 0u)) << k;
    }
    // no early exit for an octet without hits: the branch costs more than
    // the index arithmetic it would skip (almost every octet has a hit)
    int l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        l[k] = staged_index(word[k], boff[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if ((hm >> k) & 1u) atomicAdd(&cnt[TC_IX(l[k], lk.hv)], 1u);
    return hm;
}

template <bool EC>
__device__ __forceinline__ uint32_t visit_octet_bitmap(const lookup_bitmap& lk, const octet& o, int64_t pos,
                                                       int off, int len, uint32_t* cnt, int64_t h0,
                                                       ull* __restrict__ tri, uint32_t* __restrict__ flag,
                                                       const tc_dims& dm) {
    const uint32_t hm = octet_hits_bitmap(lk, o, off, len, cnt);
    mark_octet<EC>(flag, pos, hm, dm);
    return (uint32_t)__popc(hm);
}

#ifndef TC_GROUP_VALID
#define TC_GROUP_VALID 1
#endif
// The G octets of a lane (8 G ids from the 8-aligned position pos) lie in at
// most two 32-bit flag words when 8 G + 24 <= 64: their hit masks are put
// side by side and each word gets one OR.
#ifndef TC_FLAG_COMBINE
#define TC_FLAG_COMBINE 1
#endif
template <int G>
__device__ __forceinline__ uint32_t mark_group(uint32_t* __restrict__ f, int64_t pos, uint64_t hm,
                                               const tc_dims& dm) {
    static_assert(8 * G + 24 <= 64, "a lane's octets span more than two flag words");
    if (hm == 0) return 0;
    const uint64_t wm = hm << (pos & 31);
    const int64_t w0 = pos >> 5;
    if ((uint32_t)wm) flag_or(f, TC_IX(w0, dm.fw), (uint32_t)wm);
    if ((uint32_t)(wm >> 32)) flag_or(f, TC_IX(w0 + 1, dm.fw), (uint32_t)(wm >> 32));
    return (uint32_t)__popcll(hm);
}

// The filtered sorted list: the 8 filter bits first, then the bisection of
// the ids whose slot is set, one at a time per lane (a lane's candidates
// are few, so the warp runs the bisection once or twice per octet rather
// than once per id).
template <bool EC>
__device__ __forceinline__ uint32_t visit_octet_filtered(const lookup_filtered& lk, const octet& o, int64_t pos,
                                                         int off, int len, uint32_t* cnt,
                                                         uint32_t* __restrict__ flag, const tc_dims& dm) {
    uint32_t cand = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t h = filter_slot(o.x[k]);
        uint32_t bit = (lk.filt[h >> 5] >> (h & 31)) & 1u;
        if (TC_FILTER_HASHES > 1) {
            const uint32_t h2 = filter_slot2(o.x[k]);
            bit &= (lk.filt[h2 >> 5] >> (h2 & 31)) & 1u;
        }
        cand |= bit << k;
    }
    cand &= octet_valid(off, len);
    uint32_t hm = 0;
    while (cand) {
        const int k = __ffs(cand) - 1;
        cand &= cand - 1;
        int32_t w = o.x[0];
#pragma unroll
        for (int j = 1; j < 8; ++j) w = k == j ? o.x[j] : w;
        int l = 0;
        if (lk.ls.find(w, l)) {
            atomicAdd(&cnt[TC_IX(l, lk.ls.hv)], 1u);
            hm |= 1u << k;
        }
    }
    mark_octet<EC>(flag, pos, hm, dm);
    return (uint32_t)__popc(hm);
}

// The G octets of one lane at the 8-aligned position pos (the first id at
// offset off0 from its stream start, len ids in the stream).  Returns the hits.
template <class LK, bool CNT, int G, bool EC>
__device__ __forceinline__ uint32_t visit_group(const LK& lk, const octet (&o)[G], int64_t pos, int off0, int len,
                                                uint32_t* cnt, int64_t h0, ull* __restrict__ tri,
                                                uint32_t* __restrict__ flag, const tc_dims& dm) {
    uint32_t h = 0;
    if constexpr (std::is_same<LK, lookup_bitmap>::value && CNT && !EC && TC_FLAG_COMBINE && G > 1) {
        uint32_t hm = 0;
        if (TC_GROUP_VALID) {
            const uint32_t valid = group_valid<G>(off0, len);
#pragma unroll
            for (int j = 0; j < G; ++j) hm |= octet_hits_masked(lk, o[j], (valid >> (8 * j)) & 0xffu, cnt) << (8 * j);
        } else {
#pragma unroll
            for (int j = 0; j < G; ++j) hm |= octet_hits_bitmap(lk, o[j], off0 + 8 * j, len, cnt) << (8 * j);
        }
        h = mark_group<G>(flag, pos, hm, dm);
    } else {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if constexpr (std::is_same<LK, lookup_bitmap>::value && CNT)
                h += visit_octet_bitmap<EC>(lk, o[j], pos + 8 * j, off0 + 8 * j, len, cnt, h0, tri, flag, dm);
            else if constexpr (std::is_same<LK, lookup_filtered>::value)
                h += visit_octet_filtered<EC>(lk, o[j], pos + 8 * j, off0 + 8 * j, len, cnt, flag, dm);
            else
                h += visit_octet<LK, CNT, EC>(lk, o[j], pos + 8 * j, off0 + 8 * j, len, cnt, h0, tri, flag, dm);
        }
    }
    return h;
}

// Walks the groups [gb, ge) of the concatenated streams of a table (nc
// streams), one group of G octets per lane per window.  The stream of each
// lane is found from the starts of the next 32 streams that fall inside the
// current 32-group window (one warp OR-reduction); s_base is the stream
// holding the group before the window.
template <class LK, bool CNT, int N, int G, bool EC>
__device__ __forceinline__ void walk_groups(int lane, stream_table<N>& tb, int nc, int gb, int ge,
                                            const LK& lk, uint32_t* cnt, int64_t h0,
                                            const int32_t* __restrict__ col, ull* __restrict__ tri,
                                            uint32_t* __restrict__ flag, const tc_dims& dm) {
    if (gb >= ge) return;
    int s_base = -1;
    if (gb > 0) {   // last stream starting at or before group gb - 1
        s_base = 0;
#pragma unroll
        for (int step = N / 2; step; step >>= 1)
            if (s_base + step < nc && tb.gpre[s_base + step] <= gb - 1) s_base += step;
    }
    const unsigned le = FULL >> (31 - lane);
    for (int F = gb; F < ge; F += 32) {
        const int cand = s_base + 1 + lane;
        const int st = cand < nc ? tb.gpre[cand] : 0x7fffffff;
        const unsigned rel = (unsigned)(st - F);
        const unsigned smask = __reduce_or_sync(FULL, rel < 32u ? (1u << rel) : 0u);
        const int my = s_base + __popc(smask & le);
        s_base += __popc(smask);
        const int q = F + lane;
        uint32_t h = 0;
        if (q < ge) {
            const int go = q - tb.gpre[my];
            const int f = tb.fl[my];
            const int64_t pos = tb.va[my] + (int64_t)(8 * G) * go;
            const int off0 = 8 * G * go - (f & 7), len = f >> 3;
            octet o[G];
#pragma unroll
            for (int j = 0; j < G; ++j) o[j] = load8(col, TC_IX(pos + 8 * j, dm.e2 + 25));
            h = visit_group<LK, CNT, G, EC>(lk, o, pos, off0, len, cnt, h0, tri, flag, dm);
        }
        if ((smask & ~1u) == 0) {
            // the whole window lies in one stream
            const uint32_t sum = __reduce_add_sync(FULL, h);
            if (lane == 0 && sum) atomicAdd(&tb.hits[my], sum);
        } else if (h) {
            atomicAdd(&tb.hits[my], h);
        }
    }
}

// Merge-path intersection of the staged A = N_H(v) (shared, ascending)
// with streams [k0, k1) of a table in turn.  The 32 lanes split the merge
// path of A and B into equal diagonals; on ties the A element is consumed
// first, and a common id is counted when its A element is consumed while
// the current B element equals it.
template <int N, bool EC>
__device__ __forceinline__ void merge_streams(int lane, int k0, int k1, stream_table<N>& tb,
                                              const int32_t* A, int na, uint32_t* cnt,
                                              const int32_t* __restrict__ col,
                                              uint32_t* __restrict__ flag, const tc_dims& dm) {
    for (int i = k0; i < k1; ++i) {
        const int nb = tb.fl[i] >> 3;
        const int64_t p0 = tb.va[i] + (tb.fl[i] & 7);
        const int32_t* B = col + TC_IX(p0, dm.e2 + 32);
        const int L = na + nb;
        const int d0 = (int)(((int64_t)L * lane) >> 5), d1 = (int)(((int64_t)L * (lane + 1)) >> 5);
        int lo = max(0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= __ldg(B + (d0 - mid - 1))) lo = mid + 1; else hi = mid;
        }
        int ia = lo, jb = d0 - lo;
        uint32_t found = 0;
        for (int d = d0; d < d1; ++d) {
            if (ia < na && (jb >= nb || A[ia] <= __ldg(B + jb))) {
                if (jb < nb && __ldg(B + jb) == A[ia]) {
                    atomicAdd(&cnt[TC_IX(ia, na)], 1u);
                    mark<EC>(flag, p0 + jb, 1u, dm);
                    ++found;
                }
                ++ia;
            } else {
                ++jb;
            }
        }
        found = __reduce_add_sync(FULL, found);
        if (lane == 0 && found) tb.hits[i] += found;
        __syncwarp();
    }
}

// ------------------------------------------------------------ warp items
// One warp per item, N_H(v) staged in the warp's own shared region: a
// bitmap when its window fits, else a sorted list (|N_H(v)| <= TC_WARP_CAP).
constexpr int kWarpSmem = 8 * TC_WARP_CAP;
struct warp_smem {
    uint8_t region[kWarpSmem];
    uint32_t filt[kFilterWords];
    stream_table<32> tb;
};
#ifndef TC_WARP_FETCH
#define TC_WARP_FETCH 4
#endif
#ifndef TC_WARP_FILTER
#define TC_WARP_FILTER 1
#endif
constexpr int kWarpItemsPerFetch = TC_WARP_FETCH;

__device__ __forceinline__ bool warp_bitmap_fits(int64_t words, int64_t hv) {
    return hv < 65536 && bitmap_bytes(words, hv) <= kWarpSmem;
}

// Compacts a warp's 32 entries into its stream table; returns the total
// number of groups and the number of streams in nc.
template <int G>
__device__ __forceinline__ int compact_warp(int lane, const entry& e, stream_table<32>& tb, int& nc) {
    const int ng = entry_groups<G>(e);
    const unsigned nz = __ballot_sync(FULL, ng > 0);
    int incl = ng;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int x = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += x;
    }
    if (ng > 0) put_stream(e, __popc(nz & ((1u << lane) - 1)), incl - ng, tb);
    nc = __popc(nz);
    __syncwarp();
    return __shfl_sync(FULL, incl, 31);
}

#ifndef TC_WARP_G
#define TC_WARP_G 1
#endif
#ifndef TC_CTA_G
#define TC_CTA_G 3
#endif
constexpr int kWarpG = TC_WARP_G;   // octets (8 ids) per lane per window, warp items
constexpr int kCtaG = TC_CTA_G;     // octets per lane per window, CTA items

#ifndef TC_WARP_MIN_BLOCKS
#define TC_WARP_MIN_BLOCKS 4
#endif
template <bool MERGE, bool EC>
__global__ void __launch_bounds__(TC_CTA_THREADS, TC_WARP_MIN_BLOCKS)
k_count_warp(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
             const int64_t* __restrict__ hstart, const tc_head* __restrict__ head,
             const tc_item* __restrict__ it_d, const int32_t* __restrict__ it_nb,
             const int64_t* __restrict__ it_pb, const int64_t* __restrict__ it_pe,
             int64_t n_items, int64_t it_off, int64_t it_stride, ull* __restrict__ cursor, int strategy,
             ull* __restrict__ tri, uint32_t* __restrict__ flag, ull* __restrict__ total, tc_dims dm) {
    __shared__ __align__(16) warp_smem sm[kCtaWarps];
    const int lane = threadIdx.x & 31;
    warp_smem& ws = sm[threadIdx.x >> 5];
    const bool allow_bitmap = !MERGE && (strategy == TC_STRATEGY_AUTO || strategy == TC_STRATEGY_BITMAP);
    ull tv_all = 0;
    auto wbar = [] { __syncwarp(); };
    for (;;) {
        int64_t base = 0;
        if (lane == 0) base = (int64_t)atomicAdd(cursor, (ull)kWarpItemsPerFetch);
        base = __shfl_sync(FULL, base, 0);
        if (base >= n_items) break;
        const int64_t lim = min(base + kWarpItemsPerFetch, n_items);
        for (int64_t it = base; it < lim; ++it) {
            const int64_t gi = it_off + it_stride * it;   // this shard's it-th item
            const tc_item d = it_d[gi];
            const int32_t v = d.v, nbits = it_nb[gi];
            const int64_t pb = it_pb[gi], pe = it_pe[gi];
            entry nxt = fetch_entry(pb + lane, pe, head, dm);
            const int64_t h0 = d.h0;
            const int hv = d.hv;
            const bool use_bitmap = allow_bitmap && warp_bitmap_fits((nbits + 31) >> 5, hv);
            // the filter in front of the bisection: automatic strategy only,
            // so that a forced binary search still bisects every id
            const bool use_filter = !MERGE && !use_bitmap && TC_WARP_FILTER && strategy == TC_STRATEGY_AUTO;
            uint32_t* cnt;
            lookup_bitmap lb{};
            int32_t* ids = (int32_t*)ws.region;
            if (use_bitmap) {
                lb = build_bitmap(lane, 32, ws.region, v, h0, hv, nbits, col, cnt, wbar, nullptr, lane, 0, 1, dm);
            } else {
                cnt = (uint32_t*)(ids + TC_WARP_CAP);
                if (use_filter)
                    for (int i = lane; i < kFilterWords; i += 32) ws.filt[i] = 0;
                __syncwarp();
                for (int i = lane; i < hv; i += 32) {
                    const int32_t x = col[TC_IX(h0 + i, dm.e2)];
                    ids[TC_IX(i, TC_WARP_CAP)] = x;
                    cnt[TC_IX(i, TC_WARP_CAP)] = 0;
                    if (use_filter) {
                        const uint32_t h = filter_slot(x);
                        atomicOr(&ws.filt[h >> 5], 1u << (h & 31));
                        if (TC_FILTER_HASHES > 1) {
                            const uint32_t h2 = filter_slot2(x);
                            atomicOr(&ws.filt[h2 >> 5], 1u << (h2 & 31));
                        }
                    }
                }
                __syncwarp();
            }
            const lookup_sorted ls{ids, hv};
            const lookup_filtered lf{ls, ws.filt};
            ull tv = 0;
            for (int64_t b = pb; b < pe; b += 32) {
                const entry cur = nxt;
                nxt = fetch_entry(b + 32 + lane, pe, head, dm);   // in flight meanwhile
                int nc;
                const int groups = compact_warp<kWarpG>(lane, cur, ws.tb, nc);
                if (MERGE) merge_streams<32, EC>(lane, 0, nc, ws.tb, ids, hv, cnt, col, flag, dm);
                else if (use_bitmap) walk_groups<lookup_bitmap, true, 32, kWarpG, EC>(lane, ws.tb, nc, 0, groups, lb, cnt, h0, col, tri, flag, dm);
                else if (use_filter) walk_groups<lookup_filtered, true, 32, kWarpG, EC>(lane, ws.tb, nc, 0, groups, lf, cnt, h0, col, tri, flag, dm);
                else walk_groups<lookup_sorted, true, 32, kWarpG, EC>(lane, ws.tb, nc, 0, groups, ls, cnt, h0, col, tri, flag, dm);
                __syncwarp();
                if (lane < nc) close_stream<32, EC>(lane, ws.tb, tri, flag, tv, dm);
                __syncwarp();
            }
            for (int i = lane; i < hv; i += 32) {
                const uint32_t c = cnt[i];
                if (c) {
                    atomicAdd(&tri[TC_IX(col[TC_IX(h0 + i, dm.e2)], dm.n)], (ull)c);
                    mark<EC>(flag, h0 + i, c, dm);
                }
            }
            tv = warp_sum(tv);
            if (lane == 0 && tv) atomicAdd(&tri[TC_IX(v, dm.n)], tv);
            tv_all += tv;
            __syncwarp();
        }
    }
    if (lane == 0 && tv_all) atomicAdd(total, tv_all);
}

// ------------------------------------------------------------- CTA items
// One CTA of T threads per item; its T / 32 warps share the staged N_H(v).
// The item's head entries are taken in rounds of T (a stream table, the next
// round's entries loaded while this one streams); the round's units are
// split evenly over the warps.  T = 256 by default; graphs whose CTA items
// are small (a small chunk target, e.g. grids with Chung-Lu hubs) take
// T = 512, so that staging and each round are shared by twice the warps.
template <int LOOK, bool MERGE, bool EC, int T = kCtaT>
__global__ void __launch_bounds__(T, 1024 / T)
k_count_cta(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
            const int64_t* __restrict__ hstart, const tc_head* __restrict__ head,
            const tc_item* __restrict__ it_d, const int32_t* __restrict__ it_nb,
            const int64_t* __restrict__ it_pb, const int64_t* __restrict__ it_pe,
            int64_t n_items, int64_t it_off, int64_t it_stride, ull* __restrict__ cursor, int strategy,
            ull* __restrict__ tri,
            uint32_t* __restrict__ flag, ull* __restrict__ total, tc_dims dm) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ __align__(16) stream_table<T> tb;
    __shared__ int64_t s_item;
    __shared__ ull s_tv[(T / 32)];
    __shared__ uint32_t s_scan[(T / 32)];
    __shared__ int s_cnt[(T / 32)];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = threadIdx.x, nt = T;
    auto cbar = [] { __syncthreads(); };
    for (;;) {
        __syncthreads();
        if (t == 0) s_item = (int64_t)atomicAdd(cursor, 1ull);
        __syncthreads();
        const int64_t it = s_item;
        if (it >= n_items) break;
        const int64_t gi = it_off + it_stride * it;   // this shard's it-th item
        const tc_item d = it_d[gi];
        const int32_t v = d.v;
        const int64_t pb = it_pb[gi], pe = it_pe[gi];
        entry nxt = fetch_entry(pb + t, pe, head, dm);
        const int64_t h0 = d.h0;
        const int hv = d.hv;
        uint32_t* cnt = nullptr;
        lookup_bitmap lb{};
        lookup_sorted ls{};
        lookup_global lg{};
        if (LOOK == L_BITMAP) {
            lb = build_bitmap(t, nt, dyn, v, h0, hv, it_nb[gi], col, cnt, cbar, s_scan, lane, warp, (T / 32), dm);
        } else if (LOOK == L_SORTED) {
            int32_t* ids = (int32_t*)dyn;
            cnt = (uint32_t*)(ids + hv);
            for (int i = t; i < hv; i += nt) {
                ids[i] = col[TC_IX(h0 + i, dm.e2)];
                cnt[i] = 0;
            }
            __syncthreads();
            ls = lookup_sorted{ids, hv};
        } else {
            lg = lookup_global{col + h0, hv};
        }
        ull tv = 0;
        for (int64_t r0 = pb; r0 < pe; r0 += T) {
            const entry cur = nxt;
            nxt = fetch_entry(r0 + T + t, pe, head, dm);   // in flight meanwhile
            // compact the round's non-empty streams: warp scans of the group
            // counts, then the warp totals
            const int ng = entry_groups<kCtaG>(cur);
            const unsigned nz = __ballot_sync(FULL, ng > 0);
            int incl = ng;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int x = __shfl_up_sync(FULL, incl, d);
                if (lane >= d) incl += x;
            }
            if (lane == 31) {
                s_scan[warp] = (uint32_t)incl;
                s_cnt[warp] = __popc(nz);
            }
            __syncthreads();
            int before_g = 0, before_c = 0, GT = 0, NC = 0;
#pragma unroll
            for (int k = 0; k < (T / 32); ++k) {
                const int sg = (int)s_scan[k], sc = s_cnt[k];
                before_g += k < warp ? sg : 0;
                before_c += k < warp ? sc : 0;
                GT += sg;
                NC += sc;
            }
            if (ng > 0) put_stream(cur, before_c + __popc(nz & ((1u << lane) - 1)), before_g + incl - ng, tb);
            __syncthreads();
            if (MERGE) {
                merge_streams<T, EC>(lane, (NC * warp) / (T / 32), (NC * (warp + 1)) / (T / 32), tb, ls.ids, hv, cnt, col, flag, dm);
            } else {
                const int gb = (int)(((int64_t)GT * warp) / (T / 32)), ge = (int)(((int64_t)GT * (warp + 1)) / (T / 32));
                if (LOOK == L_BITMAP)
                    walk_groups<lookup_bitmap, true, T, kCtaG, EC>(lane, tb, NC, gb, ge, lb, cnt, h0, col, tri, flag, dm);
                else if (LOOK == L_SORTED)
                    walk_groups<lookup_sorted, true, T, kCtaG, EC>(lane, tb, NC, gb, ge, ls, cnt, h0, col, tri, flag, dm);
                else
                    walk_groups<lookup_global, false, T, kCtaG, EC>(lane, tb, NC, gb, ge, lg, nullptr, h0, col, tri, flag, dm);
            }
            __syncthreads();   // every group of the round is done
            // no barrier after the closes: the next round rewrites the table
            // only after its first barrier, which every thread reaches once
            // its own close is done
            if (t < NC) close_stream<T, EC>(t, tb, tri, flag, tv, dm);
        }
        tv = warp_sum(tv);
        if (lane == 0) s_tv[warp] = tv;
        __syncthreads();
        if (LOOK != L_GLOBAL) {
            for (int i = t; i < hv; i += nt) {
                const uint32_t c = cnt[i];
                if (c) {
                    atomicAdd(&tri[TC_IX(col[TC_IX(h0 + i, dm.e2)], dm.n)], (ull)c);
                    mark<EC>(flag, h0 + i, c, dm);
                }
            }
        }
        if (t == 0) {
            ull sum = 0;
            for (int k = 0; k < (T / 32); ++k) sum += s_tv[k];
            if (sum) {
                atomicAdd(&tri[TC_IX(v, dm.n)], sum);
                atomicAdd(total, sum);
            }
        }
    }
}

// ------------------------------------------------------------ thread items
// Tiny middle vertices (|N_H(v)| <= kThreadMaxH, head entries + streamed
// ids <= the planner's thread_work) take one thread each: N_H(v) is staged in the
// thread's own column of shared memory (S[k][t], so that the threads of a
// warp hit distinct banks), and every stream of the vertex is merged
// against it.  A hit at staged index a and stream position q is the
// triangle (u, v, w): △(w) += 1, edges (u, w) at q and (v, w) at h0 + a
// marked, then per stream △(u) and edge (u, v) at twin, per vertex △(v).
#ifndef TC_THREAD_MAX_H
#define TC_THREAD_MAX_H 32
#endif
#ifndef TC_THREAD_BLOCK
#define TC_THREAD_BLOCK 256
#endif
constexpr int kThreadMaxH = TC_THREAD_MAX_H;      // staged ids per thread (a column of S)
constexpr int kThreadBlock = TC_THREAD_BLOCK;     // threads of the thread-item kernel
#ifndef TC_THREAD_ILP
#define TC_THREAD_ILP 4
#endif
constexpr int kThreadILP = TC_THREAD_ILP;         // independent loads in flight per thread
// thread items at or above which those of at most 16 staged ids get their own launch
#ifndef TC_THREAD_SPLIT_ITEMS
#define TC_THREAD_SPLIT_ITEMS (8 << 20)
#endif
constexpr int64_t kThreadSplitItems = TC_THREAD_SPLIT_ITEMS;
static_assert(kThreadMaxH * kThreadBlock * 4 <= 48 * 1024, "thread-item staging exceeds static shared memory");

template <bool EC, int MAXH = kThreadMaxH, int MINH = 0>
__global__ void __launch_bounds__(kThreadBlock)
k_count_thread(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const int64_t* __restrict__ hstart, const tc_head* __restrict__ head,
               const tc_item* __restrict__ it_d, const int32_t* __restrict__ it_nb, const int64_t* __restrict__ it_pb,
               const int64_t* __restrict__ it_pe, int64_t n_items, int64_t it_off, int64_t it_stride,
               ull* __restrict__ cursor, int strategy,
               ull* __restrict__ tri, uint32_t* __restrict__ flag, ull* __restrict__ total, tc_dims dm) {
    __shared__ int32_t S[MAXH][kThreadBlock];   // items with MINH <= |N_H(v)| <= MAXH; the others skipped
    const int t = threadIdx.x;
    ull tv_all = 0;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + t; it < n_items; it += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gi = it_off + it_stride * it;   // this shard's it-th item
        const tc_item d = it_d[gi];
        if (d.hv < MINH || d.hv > MAXH) continue;   // another launch's item
        const int32_t v = d.v;
        const int64_t h0 = d.h0;
        const int hv = d.hv;
        // loads issued kThreadILP at a time, so that one thread's chain of
        // small reads does not wait for each in turn
        for (int k0 = 0; k0 < hv; k0 += kThreadILP) {
            int32_t x[kThreadILP];
#pragma unroll
            for (int j = 0; j < kThreadILP; ++j) x[j] = k0 + j < hv ? col[TC_IX(h0 + k0 + j, dm.e2)] : 0;
#pragma unroll
            for (int j = 0; j < kThreadILP; ++j)
                if (k0 + j < hv) S[TC_IX(k0 + j, MAXH)][t] = x[j];
        }
        ull tv = 0;
        const int64_t pb = it_pb[gi], pe = it_pe[gi];
        tc_head nrec{};
        if (pb < pe) nrec = head[TC_IX(pb, dm.e2)];
        for (int64_t p = pb; p < pe; ++p) {
            const tc_head rec = nrec;
            if (p + 1 < pe) nrec = head[TC_IX(p + 1, dm.e2)];   // in flight meanwhile
            const int64_t q0 = rec.twin + 1;
            const int len = rec.hrem;
            uint32_t hits = 0;
            // first staged id not below the stream's first id (bisection)
            int a = 0;
            if (len > 0) {
                const int32_t w0 = col[TC_IX(q0, dm.e2)];
                int cnt = hv;
                while (cnt > 0) {
                    const int half = cnt >> 1;
                    if (S[a + half][t] < w0) {
                        a += half + 1;
                        cnt -= half + 1;
                    } else {
                        cnt = half;
                    }
                }
            }
            for (int j0 = 0; j0 < len && a < hv; j0 += kThreadILP) {
                int32_t wv[kThreadILP];
#pragma unroll
                for (int j = 0; j < kThreadILP; ++j) wv[j] = j0 + j < len ? col[TC_IX(q0 + j0 + j, dm.e2)] : 0;
#pragma unroll
                for (int j = 0; j < kThreadILP; ++j) {
                    const int32_t w = wv[j];
                    if (j0 + j < len) {
                        while (a < hv && S[a][t] < w) ++a;
                        if (a < hv && S[a][t] == w) {
                            atomicAdd(&tri[TC_IX(w, dm.n)], 1ull);
                            mark<EC>(flag, q0 + j0 + j, 1u, dm);
                            mark<EC>(flag, h0 + a, 1u, dm);
                            ++hits;
                            ++a;
                        }
                    }
                }
            }
            if (hits) {
                atomicAdd(&tri[TC_IX(rec.u, dm.n)], (ull)hits);
                mark<EC>(flag, rec.twin, hits, dm);
                tv += hits;
            }
        }
        if (tv) atomicAdd(&tri[TC_IX(v, dm.n)], tv);
        tv_all += tv;
    }
    tv_all = warp_sum(tv_all);
    if ((t & 31) == 0 && tv_all) atomicAdd(total, tv_all);
}

// ------------------------------------------------------------ planner
struct class_acc {
    unsigned long long items[TC_NUM_CLS];
    unsigned long long staged[TC_NUM_CLS];
    unsigned long long head[TC_NUM_CLS];
    unsigned long long wedges[TC_NUM_CLS];
    unsigned long long max_bm[TC_NUM_CLS];   // largest bitmap staging of the class's items (bytes;
                                             // for the thread class: the largest |N_H(v)|)
};

// Class and chunk count of every middle vertex; rows visited in reverse
// rank order so that the heaviest vertices come first in every class.
__global__ void k_classify(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                           const int32_t* __restrict__ col, const int64_t* __restrict__ work,
                           int64_t n, int strategy, tc_plan_params pp, int64_t* __restrict__ cnt,
                           int8_t* __restrict__ cls, class_acc* __restrict__ acc) {
    ull loc[4][TC_NUM_CLS] = {};   // per-thread sums, reduced per warp at the end
    int64_t bm_s = 0, bm_l = 0;    // largest bitmap staging of this thread's small- and large-bitmap items
    int64_t hv_t = 0;              // largest |N_H(v)| of its thread items
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
            const int64_t bm = hv < 65536 ? bitmap_bytes(words, hv) : (int64_t)1 << 62;
            const bool warp_bm = bm <= kWarpSmem;
            const bool warp_list = hv <= TC_WARP_CAP;
            const bool cta_s = bm <= kBitmapSmallSmem, cta_l = bm <= kBitmapLargeSmem;
            if (strategy == TC_STRATEGY_GLOBAL) {
                c = TC_CLS_CTA_LIST;
            } else if (strategy == TC_STRATEGY_BSEARCH || strategy == TC_STRATEGY_MERGE) {
                c = warp_list ? TC_CLS_WARP : TC_CLS_CTA_LIST;
            } else if (strategy == TC_STRATEGY_BITMAP) {
                c = warp_bm ? TC_CLS_WARP : cta_s ? TC_CLS_BITMAP_S : cta_l ? TC_CLS_BITMAP_L
                  : warp_list ? TC_CLS_WARP : TC_CLS_CTA_LIST;
            } else {
                // AUTO: tiny vertices one per thread; heavy vertices on a CTA
                // bitmap when zeroing it is cheap next to the work; the rest
                // on a warp (bitmap or list)
                const bool heavy = W >= pp.cta_min_work && W >= 2 * words;
                if (hv <= kThreadMaxH && lv + W <= pp.thread_work) c = TC_CLS_THREAD;
                else if (heavy && cta_s) c = TC_CLS_BITMAP_S;
                else if (heavy && cta_l) c = TC_CLS_BITMAP_L;
                else if (warp_bm || warp_list) c = TC_CLS_WARP;
                else if (cta_s) c = TC_CLS_BITMAP_S;
                else if (cta_l) c = TC_CLS_BITMAP_L;
                else c = TC_CLS_CTA_LIST;
            }
            const int64_t chunk = c == TC_CLS_WARP ? pp.warp_chunk : pp.cta_chunk;
            chunks = c == TC_CLS_THREAD ? 1 : (W + chunk - 1) / chunk;
            if (chunks > lv) chunks = lv;
            if (chunks < 1) chunks = 1;
#pragma unroll
            for (int cc = 0; cc < TC_NUM_CLS; ++cc)   // static indices keep loc in registers
                if (cc == c) {
                    loc[0][cc] += (ull)chunks;
                    loc[1][cc] += (ull)hv;
                    loc[2][cc] += (ull)lv;
                    loc[3][cc] += (ull)W;
                }
            if (c == TC_CLS_THREAD) hv_t = hv > hv_t ? hv : hv_t;
            if (c == TC_CLS_BITMAP_S) bm_s = bm > bm_s ? bm : bm_s;
            if (c == TC_CLS_BITMAP_L) bm_l = bm > bm_l ? bm : bm_l;
        }
        cls[i] = (int8_t)c;
        for (int k = 0; k < TC_NUM_CLS; ++k) cnt[k * (n + 1) + i] = (k == c) ? chunks : 0;
    }
    const int lane = threadIdx.x & 31;
    for (int o = 16; o; o >>= 1) {
        const int64_t x = __shfl_xor_sync(0xffffffffu, bm_s, o), y = __shfl_xor_sync(0xffffffffu, bm_l, o);
        const int64_t z = __shfl_xor_sync(0xffffffffu, hv_t, o);
        bm_s = x > bm_s ? x : bm_s;
        bm_l = y > bm_l ? y : bm_l;
        hv_t = z > hv_t ? z : hv_t;
    }
    if (lane == 0) {
        if (bm_s) atomicMax(&acc->max_bm[TC_CLS_BITMAP_S], (ull)bm_s);
        if (bm_l) atomicMax(&acc->max_bm[TC_CLS_BITMAP_L], (ull)bm_l);
        if (hv_t) atomicMax(&acc->max_bm[TC_CLS_THREAD], (ull)hv_t);   // for this class: staged ids
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < TC_NUM_CLS; ++c) {
            ull x = loc[a][c];
            for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0 && x) {
                ull* dst = a == 0 ? acc->items : a == 1 ? acc->staged : a == 2 ? acc->head : acc->wedges;
                atomicAdd(&dst[c], x);
            }
        }
}

struct emit_targets {
    tc_item* d[TC_NUM_CLS];
    int32_t* nb[TC_NUM_CLS];
    int64_t* pb[TC_NUM_CLS];
    int64_t* pe[TC_NUM_CLS];
};

__global__ void k_emit(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                       const int32_t* __restrict__ col,
                       int64_t n, const int8_t* __restrict__ cls, const int64_t* __restrict__ cnt,
                       const int64_t* __restrict__ off, emit_targets tg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cls[i];
        if (c < 0) continue;
        const int64_t r = n - 1 - i;
        const int64_t b = row_ptr[r], h0 = hstart[r], lv = h0 - b, h1 = row_ptr[r + 1];
        const int64_t k = cnt[c * (n + 1) + i], o = off[c * (n + 1) + i];
        const tc_item d{h0, (int32_t)r, (int32_t)(h1 - h0)};
        const int32_t nbits = h1 > h0 ? col[h1 - 1] - (int32_t)r : 0;
        tc_item* dd = tg.d[c];
        int32_t* nbb = tg.nb[c];
        int64_t* pbb = tg.pb[c];
        int64_t* pee = tg.pe[c];
        for (int64_t j = 0; j < k; ++j) {
            dd[o + j] = d;
            nbb[o + j] = nbits;
            pbb[o + j] = b + lv * j / k;
            pee[o + j] = b + lv * (j + 1) / k;
        }
    }
}

inline int blocks_for(int64_t items) {
    int64_t b = (items + 255) / 256, cap = (int64_t)sm_count() * 16;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

// Per-kernel launch shape, computed once (so that later launches, e.g.
// inside a stream capture, make no attribute or occupancy calls).  One
// kernel may be launched with several dynamic shared sizes (the bitmap
// kernel serves both bitmap classes), and its maximum-dynamic-shared
// attribute is one value per kernel: it is only ever raised, so a launch
// with a smaller size never lowers it below what a larger one needs.
struct launch_shape {
    const void* fn;
    size_t smem;
    int per_sm;
};
struct smem_attr {
    const void* fn;
    size_t max_smem;
};
std::mutex g_shape_mu;
launch_shape g_shapes[32];
int g_nshapes = 0;
smem_attr g_attrs[16];
int g_nattrs = 0;

tc_status shape_for(const void* fn, size_t smem, int threads, int& per_sm) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    for (int i = 0; i < g_nshapes; ++i)
        if (g_shapes[i].fn == fn && g_shapes[i].smem == smem) {
            per_sm = g_shapes[i].per_sm;
            return TC_OK;
        }
    // static + dynamic shared memory may exceed the 48 KB default
    if (smem > 0) {
        int a = 0;
        while (a < g_nattrs && g_attrs[a].fn != fn) ++a;
        if (a == g_nattrs || g_attrs[a].max_smem < smem) {
            TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            if (a == g_nattrs && g_nattrs < 16) g_attrs[g_nattrs++] = smem_attr{fn, smem};
            else if (a < g_nattrs) g_attrs[a].max_smem = smem;
        }
    }
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    per_sm = std::max(per_sm, 1);
    if (g_nshapes < 32) g_shapes[g_nshapes++] = launch_shape{fn, smem, per_sm};
    return TC_OK;
}

template <class K>
tc_status launch_persistent(K kernel, const char* name, size_t smem, int64_t all_items, cudaStream_t s,
                            const tc_graph* g, const tc_plan& p, int c, ull* cursor, uint32_t* marks,
                            int shard, int num_shards, int threads = TC_CTA_THREADS) {
    // shard k of K takes items k, k + K, k + 2K, ... of the class (heaviest
    // first, so the shards' work comes out close to equal)
    const int64_t items = all_items > shard ? (all_items - shard + num_shards - 1) / num_shards : 0;
    if (items == 0) return TC_OK;
    int per_sm = 1;
    TC_TRY(shape_for((const void*)kernel, smem, threads, per_sm));
    int64_t blocks = std::min<int64_t>((int64_t)sm_count() * per_sm, items);
    launch_scope ls(name, s);
    kernel<<<(int)blocks, threads, smem, s>>>(g->row_ptr, g->col, g->hstart, g->head,
                                                     p.d[c], p.nb[c], p.pb[c], p.pe[c], items, (int64_t)shard,
                                                     (int64_t)num_shards, cursor,
                                                     g->strategy, g->tri, marks, g->counters, dims_of(g));
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

void free_plan(tc_plan& p, cudaStream_t s) {
    for (int c = 0; c < TC_NUM_CLS; ++c) {
        dfree(p.d[c], s);
        dfree(p.nb[c], s);
        dfree(p.pb[c], s);
        dfree(p.pe[c], s);
        p.d[c] = nullptr;
        p.nb[c] = nullptr;
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
            free_plan(p, s);     \
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
                                                  g->params, cnt, cls, acc);
        PLAN_CUDA(cudaGetLastError());
    }
    PLAN_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, cnt, off, n + 1, s));
    PLAN_TRY(dalloc((void**)&tmp, tmp_bytes, s));
    {
        launch_scope ls("plan_scan", s);
        for (int c = 0; c < TC_NUM_CLS; ++c)
            PLAN_TRY(run_library("scan_plan", n + 1, 0, c == 0, s, [&](cudaStream_t st) {
                return cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt + c * (n + 1), off + c * (n + 1),
                                                     n + 1, st);
            }));
    }
    class_acc h{};
    PLAN_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    PLAN_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < TC_NUM_CLS; ++c) {
        p.count[c] = (int64_t)h.items[c];
        PLAN_TRY(dalloc((void**)&p.d[c], (p.count[c] + 1) * sizeof(tc_item), s));
        PLAN_TRY(dalloc((void**)&p.nb[c], (p.count[c] + 1) * 4, s));
        PLAN_TRY(dalloc((void**)&p.pb[c], (p.count[c] + 1) * 8, s));
        PLAN_TRY(dalloc((void**)&p.pe[c], (p.count[c] + 1) * 8, s));
    }
    if (n > 0) {
        launch_scope ls("plan_emit", s);
        emit_targets tg;
        for (int c = 0; c < TC_NUM_CLS; ++c) {
            tg.d[c] = p.d[c];
            tg.nb[c] = p.nb[c];
            tg.pb[c] = p.pb[c];
            tg.pe[c] = p.pe[c];
        }
        k_emit<<<blocks_for(n), 256, 0, s>>>(g->row_ptr, g->hstart, g->col, n, cls, cnt, off, tg);
        PLAN_CUDA(cudaGetLastError());
    }
    // the bitmap kernels get the shared memory their largest item needs, not
    // the class limit: what they leave is L1, which the id streams use (the
    // large-bitmap kernel at R-MAT scale 24: 2.14 -> 1.88 ms with 28 KB
    // more L1 per SM)
    auto tight = [](unsigned long long need, int64_t cap) {
        const int64_t kb = ((int64_t)need + 1023) / 1024 * 1024;
        return (size_t)(TC_TIGHT_SMEM && kb > 0 && kb < cap ? kb : cap);
    };
    p.smem[TC_CLS_BITMAP_S] = tight(h.max_bm[TC_CLS_BITMAP_S], kBitmapSmallSmem);
    p.smem[TC_CLS_BITMAP_L] = tight(h.max_bm[TC_CLS_BITMAP_L], kBitmapLargeSmem);
    p.smem[TC_CLS_WARP] = 0;
    p.smem[TC_CLS_CTA_LIST] = kCtaListSmem;
    p.smem[TC_CLS_THREAD] = 0;
    p.thread_max_h = (int)h.max_bm[TC_CLS_THREAD];
    p.strategy = strategy;
    g->plan_params_version = g->params_version;
    // algorithmic bytes of each class's kernel: stage N_H(v) once (4 hv),
    // read each head entry's label, twin and stream length (16), stream each
    // wedge id (4)
    tc_graph_stats& S = g->stats;
    for (int c = 0; c < TC_NUM_CLS; ++c) {
        S.items[c] = p.count[c];
        S.class_bytes[c] = 4.0 * (double)h.staged[c] + 16.0 * (double)h.head[c] + 4.0 * (double)h.wedges[c];
        S.class_wedges[c] = (double)h.wedges[c];
        S.class_head[c] = (double)h.head[c];
    }
    cleanup();
    PLAN_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
#undef PLAN_TRY
#undef PLAN_CUDA
}

namespace {

// Flag bits from per-entry triangle counts (edge-count mode): each warp
// turns 32 consecutive counts into one flag word.
__global__ void k_flags_from_counts(const uint32_t* __restrict__ ecnt, int64_t e2, uint32_t* __restrict__ flag) {
    const int64_t words = (e2 + 31) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < (words << 5); p += stride) {
        const unsigned bits = __ballot_sync(0xffffffffu, p < e2 && ecnt[p] != 0);
        if ((threadIdx.x & 31) == 0) flag[p >> 5] = bits;
    }
}

template <bool EC>
tc_status launch_count_kernels(tc_graph* g, cudaStream_t s, uint32_t* marks, int shard, int num_shards) {
    const tc_plan& p = g->plan;
    ull* cur = g->counters + 1;
    const bool merge = g->strategy == TC_STRATEGY_MERGE;
    const char* nm[5] = {EC ? "count_edges_bitmap_l" : "count_bitmap_l", EC ? "count_edges_bitmap_s" : "count_bitmap_s",
                         EC ? "count_edges_cta_list" : "count_cta_list", EC ? "count_edges_cta_global" : "count_cta_global",
                         EC ? "count_edges_warp" : "count_warp"};
    // thread items stage N_H(v) in a column of shared memory.  Unions of
    // many small graphs (millions of thread items, nearly all with at most
    // 16 ids) run those in a launch that holds half of it, the rest going
    // to L1, and the others, if any, in a second launch over the same list
    // (the 8192-graph batch: 5.0 -> 3.9 ms); with fewer items the second
    // pass over the list costs more than it saves
    const bool split = p.thread_max_h <= 16 || p.count[TC_CLS_THREAD] >= kThreadSplitItems;
    if (split)
        TC_TRY(launch_persistent(k_count_thread<EC, 16, 0>, EC ? "count_edges_thread" : "count_thread", 0,
                                 p.count[TC_CLS_THREAD], s, g, p, TC_CLS_THREAD, cur + TC_CLS_THREAD, marks, shard,
                                 num_shards, kThreadBlock));
    if (split && p.thread_max_h > 16)
        TC_TRY(launch_persistent(k_count_thread<EC, kThreadMaxH, 17>, EC ? "count_edges_thread" : "count_thread",
                                 0, p.count[TC_CLS_THREAD], s, g, p, TC_CLS_THREAD, cur + TC_CLS_THREAD, marks,
                                 shard, num_shards, kThreadBlock));
    else if (!split)
        TC_TRY(launch_persistent(k_count_thread<EC, kThreadMaxH, 0>, EC ? "count_edges_thread" : "count_thread",
                                 0, p.count[TC_CLS_THREAD], s, g, p, TC_CLS_THREAD, cur + TC_CLS_THREAD, marks,
                                 shard, num_shards, kThreadBlock));
    // heaviest classes first; each kernel drains its own item queue
    if (TC_WIDE_L)
        TC_TRY(launch_persistent(k_count_cta<L_BITMAP, false, EC, 2 * kCtaT>, nm[0], p.smem[TC_CLS_BITMAP_L],
                                 p.count[TC_CLS_BITMAP_L], s, g, p, TC_CLS_BITMAP_L, cur + TC_CLS_BITMAP_L, marks,
                                 shard, num_shards, 2 * kCtaT));
    else
        TC_TRY(launch_persistent(k_count_cta<L_BITMAP, false, EC>, nm[0], p.smem[TC_CLS_BITMAP_L],
                                 p.count[TC_CLS_BITMAP_L], s, g, p, TC_CLS_BITMAP_L, cur + TC_CLS_BITMAP_L, marks,
                                 shard, num_shards, kCtaT));
    // small CTA items (grids with Chung-Lu hubs: 2^16-wedge chunks) share
    // their staging and rounds over 16 warps (the 4096^2 grid's bitmap
    // kernel 2.17 -> 1.47 ms); R-MAT's larger items keep 8 (16 were 20 %
    // slower at scale 22, chunks of 2^18.8 wedges, and 8 % at scale 24)
    if (g->params.cta_chunk < kWideCtaChunk)
        TC_TRY(launch_persistent(k_count_cta<L_BITMAP, false, EC, 2 * kCtaT>, nm[1], p.smem[TC_CLS_BITMAP_S],
                                 p.count[TC_CLS_BITMAP_S], s, g, p, TC_CLS_BITMAP_S, cur + TC_CLS_BITMAP_S, marks,
                                 shard, num_shards, 2 * kCtaT));
    else
        TC_TRY(launch_persistent(k_count_cta<L_BITMAP, false, EC>, nm[1], p.smem[TC_CLS_BITMAP_S],
                                 p.count[TC_CLS_BITMAP_S], s, g, p, TC_CLS_BITMAP_S, cur + TC_CLS_BITMAP_S, marks,
                                 shard, num_shards, kCtaT));
    if (p.count[TC_CLS_CTA_LIST] > 0) {
        // lists longer than the shared budget are searched in place
        const bool fits = g->strategy != TC_STRATEGY_GLOBAL &&
                          (int64_t)g->stats.max_out_degree * 8 <= (int64_t)p.smem[TC_CLS_CTA_LIST];
        if (fits && merge)
            TC_TRY(launch_persistent(k_count_cta<L_SORTED, true, EC>, nm[2], p.smem[TC_CLS_CTA_LIST],
                                     p.count[TC_CLS_CTA_LIST], s, g, p, TC_CLS_CTA_LIST, cur + TC_CLS_CTA_LIST,
                                     marks, shard, num_shards, kCtaT));
        else if (fits)
            TC_TRY(launch_persistent(k_count_cta<L_SORTED, false, EC>, nm[2], p.smem[TC_CLS_CTA_LIST],
                                     p.count[TC_CLS_CTA_LIST], s, g, p, TC_CLS_CTA_LIST, cur + TC_CLS_CTA_LIST,
                                     marks, shard, num_shards, kCtaT));
        else
            TC_TRY(launch_persistent(k_count_cta<L_GLOBAL, false, EC>, nm[3], 0, p.count[TC_CLS_CTA_LIST], s, g,
                                     p, TC_CLS_CTA_LIST, cur + TC_CLS_CTA_LIST, marks, shard, num_shards, kCtaT));
    }
    if (merge)
        TC_TRY(launch_persistent(k_count_warp<true, EC>, nm[4], 0, p.count[TC_CLS_WARP], s, g, p, TC_CLS_WARP,
                                 cur + TC_CLS_WARP, marks, shard, num_shards));
    else
        TC_TRY(launch_persistent(k_count_warp<false, EC>, nm[4], 0, p.count[TC_CLS_WARP], s, g, p, TC_CLS_WARP,
                                 cur + TC_CLS_WARP, marks, shard, num_shards));
    return TC_OK;
}

}  // namespace

tc_status run_count(tc_graph* g, cudaStream_t s, bool edge_counts, int shard, int num_shards) {
    const int64_t n = g->n, e2 = 2 * g->m;
    if (g->plan.strategy != g->strategy || g->plan_params_version != g->params_version)
        TC_TRY(make_plan(g, g->strategy, s));
    TC_CUDA(cudaMemsetAsync(g->tri, 0, (n + 1) * 8, s));
    TC_CUDA(cudaMemsetAsync(g->flag, 0, flag_words(e2) * 4, s));
    TC_CUDA(cudaMemsetAsync(g->counters, 0, 8 * 8, s));
    if (!edge_counts) {
        TC_TRY(launch_count_kernels<false>(g, s, g->flag, shard, num_shards));
        return shard == 0 ? run_core(g, s, false) : TC_OK;   // the core's triangles, once
    }
    if (!g->ecnt) TC_TRY(dalloc((void**)&g->ecnt, (e2 + 1) * 4, s));
    TC_CUDA(cudaMemsetAsync(g->ecnt, 0, (e2 + 1) * 4, s));
    TC_TRY(launch_count_kernels<true>(g, s, g->ecnt, shard, num_shards));
    if (shard == 0) TC_TRY(run_core(g, s, true));
    if (e2 > 0) {
        launch_scope ls("count_edges_flags", s);
        const int64_t words = (e2 + 31) >> 5;
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((words * 32 + 255) / 256, (int64_t)sm_count() * 16));
        k_flags_from_counts<<<blocks, 256, 0, s>>>(g->ecnt, e2, g->flag);
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}

}  // namespace tcx
