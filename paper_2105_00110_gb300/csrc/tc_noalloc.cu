// tc_csr_centrality_noalloc: triangle counts, exact numerators and TC for a
// small graph handed over as a device CSR, with every piece of working
// memory taken from one fixed array compiled into this library.
//
// The other entry points draw their working memory (CSR copies, plans, sort
// buffers) from a stream-ordered device pool.  Some callers cannot let a
// library do that: a runtime that owns all device memory through its own
// allocator and forbids hidden allocations, a latency-critical loop where a
// pool growth would stall the device, or a program whose footprint must be
// fixed before it starts.  This variant serves them for graphs up to the
// sizes stated in tc.h.  It computes the same quantities as tc_count
// followed by tc_centrality (Definition 1 through the numerator
// numer(v) = △(v) + Σ_{u∈N(v)} (u ∈ N△(v) ? 1 : 3)·△(u) of Algorithm 2 and
// one division by 3△(G)), with simpler kernels: each triangle v < u < w
// (vertex ids, no degree order) is found once from its edge (v, u) by
// looking each later neighbour w of v up in the sorted row of u.
#include <algorithm>
#include <mutex>

#include "tc_internal.cuh"

namespace {

typedef unsigned long long ull;

constexpr int64_t kMaxN = TC_NOALLOC_MAX_VERTICES;
constexpr int64_t kMaxNnz = TC_NOALLOC_MAX_ENTRIES;
constexpr int64_t kFlagWords = kMaxNnz / 64;          // one bit per CSR entry
constexpr int64_t kTriOff = 0;                        // △(v), kMaxN words
constexpr int64_t kFlagOff = kTriOff + kMaxN;         // edge flags, kFlagWords words
constexpr int64_t kDenOff = kFlagOff + kFlagWords;    // Σ_v △(v) = 3△(G)
constexpr int64_t kErrOff = kDenOff + 1;              // nonzero: the input broke a rule
constexpr int64_t kWords = (kErrOff + 1 + 31) / 32 * 32;   // 786,688 bytes

}  // namespace

// The whole working set, 768 KB per device, allocated when the module is
// loaded.  Every word a call uses (counts, flags, 3△(G), error word) is
// cleared by k_na_clear at the start of that call, so nothing carries over
// from one call to the next.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kWords];

namespace {

// Device address of g_noalloc_scratch per device, looked up once.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
ull* g_scratch_ptr[kMaxDevices] = {};

tc_status scratch_for_current_device(ull** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return tcx::from_cuda(e);
    if (dev < 0 || dev >= kMaxDevices) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return tcx::from_cuda(e);
        if (!p) return TC_ERR_CUDA;
        g_scratch_ptr[dev] = (ull*)p;
    }
    *out = g_scratch_ptr[dev];
    return TC_OK;
}

struct na_args {
    const int64_t* row_ptr;
    const int32_t* col;
    int64_t n, nnz;
    ull* tri;
    ull* flag;
    ull* den;
    ull* err;
};

__device__ __forceinline__ void na_fail(const na_args& a) { atomicOr(a.err, 1ull); }

// Row [b, e) of x, or false (and the error word set) if row_ptr breaks
// 0 = row_ptr[0] <= ... <= row_ptr[n] = nnz at x.
__device__ __forceinline__ bool na_row(const na_args& a, int64_t x, int64_t& b, int64_t& e) {
    b = a.row_ptr[x];
    e = a.row_ptr[x + 1];
    bool ok = 0 <= b && b <= e && e <= a.nnz && (x != 0 || b == 0) && (x != a.n - 1 || e == a.nnz);
    if (!ok) na_fail(a);
    return ok;
}

// Position of key in the sorted row [b, e) of col, or -1.
__device__ __forceinline__ int64_t na_find(const int32_t* col, int64_t b, int64_t e, int32_t key) {
    while (b < e) {
        const int64_t mid = b + ((e - b) >> 1);
        const int32_t c = col[mid];
        if (c == key) return mid;
        if (c < key) b = mid + 1;
        else e = mid;
    }
    return -1;
}

__device__ __forceinline__ void na_flag(const na_args& a, int64_t pos) {
    ull* w = a.flag + (pos >> 6);
    const ull bit = 1ull << (pos & 63);
    if (!(*(volatile ull*)w & bit)) atomicOr(w, bit);
}

__device__ __forceinline__ bool na_flag_get(const na_args& a, int64_t pos) {
    return (a.flag[pos >> 6] >> (pos & 63)) & 1ull;
}

__global__ void k_na_clear(ull* scratch, int64_t n, int64_t nnz) {
    const int64_t flag_words = (nnz + 63) / 64;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + flag_words + 2; i += stride) {
        if (i < n) scratch[kTriOff + i] = 0;
        else if (i < n + flag_words) scratch[kFlagOff + (i - n)] = 0;
        else scratch[kDenOff + (i - n - flag_words)] = 0;   // den, err
    }
}

// One warp per vertex v.  First the row is checked (ids in range, strictly
// increasing: sorted, no duplicates).  Then for each neighbour u > v at
// position p, each later entry w of row v (w > u) is looked up in row u;
// a hit at position q is the triangle v < u < w, whose three edges sit at
// p and the hit's position in row v (row of their lower end v) and at q
// (row of their lower end u).  Every edge's flag lives at its position in
// the row of its lower end.
__global__ void k_na_count(na_args a) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.n; v += warps) {
        int64_t b, e;
        if (!na_row(a, v, b, e)) continue;
        bool bad = false;
        for (int64_t i = b + lane; i < e; i += 32) {
            const int32_t c = a.col[i];
            if (c < 0 || c >= a.n || (i > b && a.col[i - 1] >= c)) bad = true;
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) na_fail(a);
            continue;
        }
        for (int64_t p = b; p < e; ++p) {
            const int32_t u = a.col[p];
            if (u <= v) continue;
            int64_t ub, ue;
            if (!na_row(a, u, ub, ue)) break;
            ull hits = 0;
            for (int64_t i = p + 1 + lane; i < e; i += 32) {
                const int32_t w = a.col[i];
                const int64_t q = na_find(a.col, ub, ue, w);
                if (q >= 0) {
                    ++hits;
                    atomicAdd(a.tri + w, 1ull);
                    na_flag(a, i);
                    na_flag(a, q);
                }
            }
            for (int o = 16; o; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
            if (lane == 0 && hits) {
                atomicAdd(a.tri + v, hits);
                atomicAdd(a.tri + u, hits);
                atomicAdd(a.den, 3 * hits);
                na_flag(a, p);
            }
        }
    }
}

// One warp per vertex v: numer(v) = △(v) + Σ_{u∈N(v)} (flag ? 1 : 3)·△(u),
// with the flag of (v, u) at position p of row v if u > v, else at the
// position of v in row u.  Every entry u of row v, above or below v, has
// its reverse entry v looked up in row u: a missing one means the CSR is
// not symmetric, which the count pass alone cannot see (it only follows
// entries above their row).  Then TC(v) = numer(v) / 3△(G): both operands
// stay below 2^53 within the size limits, so one IEEE division is
// correctly rounded.
__global__ void k_na_gather(na_args a, ull* d_tri, ull* d_numer, double* d_tc) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const ull den = *a.den;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < a.n; v += warps) {
        int64_t b, e;
        if (!na_row(a, v, b, e)) continue;
        ull acc = 0;
        bool bad = false;
        for (int64_t p = b + lane; p < e; p += 32) {
            const int32_t u = a.col[p];
            if (u < 0 || u >= a.n || u == v) {
                bad = true;
                continue;
            }
            int64_t ub, ue;
            if (!na_row(a, u, ub, ue)) {
                bad = true;
                continue;
            }
            const int64_t back = na_find(a.col, ub, ue, (int32_t)v);   // v's entry in row u
            if (back < 0) {
                bad = true;
                continue;
            }
            const int64_t pos = u > v ? p : back;   // the edge's flag sits in its lower end's row
            acc += (na_flag_get(a, pos) ? 1ull : 3ull) * a.tri[u];
        }
        if (bad) na_fail(a);
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const ull t = a.tri[v];
            acc += t;
            if (d_tri) d_tri[v] = t;
            if (d_numer) d_numer[v] = acc;
            if (d_tc)
                d_tc[v] = den == 0 ? __longlong_as_double(0x7ff8000000000000ll)
                                   : __ddiv_rn((double)acc, (double)den);
        }
    }
}

// If any check failed, every output is overwritten with its error marker.
__global__ void k_na_mark(const ull* err, int64_t n, ull* d_tri, ull* d_numer, double* d_tc) {
    if (*err == 0) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (d_tri) d_tri[i] = ~0ull;
        if (d_numer) d_numer[i] = ~0ull;
        if (d_tc) d_tc[i] = __longlong_as_double(0x7ff8000000000000ll);
    }
}

}  // namespace

extern "C" tc_status tc_csr_centrality_noalloc(const int64_t* d_row_ptr, const int32_t* d_col, int64_t n,
                                               int64_t nnz, uint64_t* d_tri, uint64_t* d_numer,
                                               double* d_tc, tc_stream stream) {
    tcx::nvtx_range nr("tc_csr_centrality_noalloc");
    if (n < 0 || n > kMaxN || nnz < 0 || nnz > kMaxNnz || (nnz & 1)) return TC_ERR_INVALID_ARG;
    if (n == 0 && nnz != 0) return TC_ERR_INVALID_ARG;
    if (n > 0 && !d_row_ptr) return TC_ERR_INVALID_ARG;
    if (nnz > 0 && !d_col) return TC_ERR_INVALID_ARG;
    ull* scratch = nullptr;
    TC_TRY(scratch_for_current_device(&scratch));
    if (n == 0) return TC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    na_args a{d_row_ptr, d_col, n, nnz, scratch + kTriOff, scratch + kFlagOff, scratch + kDenOff,
              scratch + kErrOff};
    const int sms = tcx::sm_count();
    const int row_blocks = (int)std::min<int64_t>((n + 7) / 8, (int64_t)sms * 8);
    const int flat_blocks = (int)std::min<int64_t>((n + (nnz + 63) / 64 + 2 + 255) / 256, (int64_t)sms * 4);
    k_na_clear<<<flat_blocks, 256, 0, s>>>(scratch, n, nnz);
    TC_LAUNCH_CHECK();
    k_na_count<<<row_blocks, 256, 0, s>>>(a);
    TC_LAUNCH_CHECK();
    k_na_gather<<<row_blocks, 256, 0, s>>>(a, (ull*)d_tri, (ull*)d_numer, d_tc);
    TC_LAUNCH_CHECK();
    k_na_mark<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 4), 256, 0, s>>>(
        scratch + kErrOff, n, (ull*)d_tri, (ull*)d_numer, d_tc);
    TC_LAUNCH_CHECK();
    tcx::add_launches(4);
    return TC_OK;
}
