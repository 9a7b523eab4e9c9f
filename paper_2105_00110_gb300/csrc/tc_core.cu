// Dense core of the count step.
//
// In degree order the highest ranks hold the hubs, and among the top C of
// them the adjacency is dense (R-MAT scale 24: density 0.13 at C = 16384).
// A triangle u < v < w whose lowest vertex u is in that core has all three
// vertices there, and the count of such triangles on each core edge (v, w)
// is the entry (A_c²)_{vw} of the core adjacency A_c: the product
// A_c² ∘ A_c restricted to the core (the matrix form of Section "Notation",
// T = A² ∘ A).  The sparse count kernels skip exactly these triangles (their
// head entries (u, v) with u in the core stream nothing) and this file adds
// them from one dense product on the tensor cores:
//
//   A_c (C x C, 0/1 in bf16)  ->  M = A_c · A_c (fp32 accumulation: exact,
//   every entry is a count of at most C ones)  ->  for every core edge (v, w)
//   with T = M_{vw}: △(v) and △(w) gain T/2 each once summed (each core
//   triangle is counted on two edges at every vertex), △(G) gains ΣT / 3, and
//   the edge is flagged when T > 0 (or t(v, w) gains T in edge-count mode).
//
// The product is a plain GEMM and goes to cuBLAS; the fill, the masked
// epilogue and the choice of C are this file's own.
#include <cublas_v2.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "tc_internal.cuh"

namespace tcx {

// -1: choose C from the graph (default), 0: never, > 0: the top C ranks.
std::atomic<long long> g_core_mode{-1};

namespace {

typedef unsigned long long ull;

constexpr int kCoreThreads = 256;
constexpr uint16_t kBf16One = 0x3F80;   // 1.0 in bfloat16
constexpr int kCoreSizes[] = {4096, 8192, 16384};
constexpr int64_t kCoreMax = 16384;

// Rough rates of the two ways to count the core's triangles, used only to
// decide whether the dense product pays: ids streamed per ms by the bitmap
// count kernel, bf16 tensor FLOP per ms of a cuBLAS GEMM, and the bytes per
// ms of the fill and the masked pass over M.  Both are below what R-MAT
// scale 24 showed (about 1.0e9 core ids/ms saved, 2.2e12 FLOP/ms), so the
// rule errs towards streaming.
constexpr double kStreamIdsPerMs = 0.7e9;
constexpr double kGemmFlopPerMs = 1.5e12;
constexpr double kPassBytesPerMs = 4.0e9;
constexpr double kMinGainMs = 0.5;

// A_c: every edge with both ends in the core, both ways (row r's N_H lies
// above r, so inside the core too).
__global__ void k_core_fill(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                            const int32_t* __restrict__ col, int64_t t, int64_t C, uint16_t* __restrict__ A) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < C; i += warps) {
        const int64_t r = t + i;
        for (int64_t p = hstart[r] + lane; p < row_ptr[r + 1]; p += 32) {
            const int64_t j = (int64_t)col[p] - t;
            A[i * C + j] = kBf16One;
            A[j * C + i] = kBf16One;
        }
    }
}

// Every core edge (tail entry p of core row r): T = M_{rw} triangles with a
// third core vertex.  S collects Σ_e T over the edges at each core vertex.
__global__ void k_core_edges(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ hstart,
                             const int32_t* __restrict__ col, int64_t t, int64_t C, const float* __restrict__ M,
                             ull* __restrict__ S, uint32_t* __restrict__ flag, uint32_t* __restrict__ ecnt,
                             ull* __restrict__ sum_t) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    ull all = 0;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < C; i += warps) {
        const int64_t r = t + i;
        ull mine = 0;
        for (int64_t p = hstart[r] + lane; p < row_ptr[r + 1]; p += 32) {
            const int64_t j = (int64_t)col[p] - t;
            const uint32_t T = (uint32_t)M[i * C + j];
            if (T) {
                mine += T;
                atomicAdd(&S[j], (ull)T);
                if (ecnt) atomicAdd(&ecnt[p], T);
                else flag_set(flag, p);
            }
        }
        for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if (lane == 0 && mine) atomicAdd(&S[i], mine);
        all += mine;
    }
    if (lane == 0 && all) atomicAdd(sum_t, all);
}

__global__ void k_core_finish(ull* __restrict__ tri, const ull* __restrict__ S, int64_t t, int64_t C,
                              const ull* __restrict__ sum_t, ull* __restrict__ total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C; i += (int64_t)gridDim.x * blockDim.x)
        tri[t + i] += S[i] >> 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(total, *sum_t / 3);
}

int warp_blocks(int64_t rows) {
    const int64_t per = kCoreThreads / 32;
    return (int)std::max<int64_t>(1, std::min<int64_t>((rows + per - 1) / per, (int64_t)sm_count() * 16));
}

// One cuBLAS handle per host thread and device, with a fixed workspace so
// that a call never allocates (and can be captured).
constexpr size_t kBlasWorkspace = 32u << 20;
struct blas_ctx {
    cublasHandle_t h = nullptr;
    void* ws = nullptr;
};
constexpr int kMaxDevices = 64;
thread_local blas_ctx t_blas[kMaxDevices];

tc_status blas_on(cudaStream_t s, cublasHandle_t* out) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return TC_ERR_INVALID_ARG;
    blas_ctx& b = t_blas[dev];
    if (!b.h) {
        if (cublasCreate(&b.h) != CUBLAS_STATUS_SUCCESS) {
            b.h = nullptr;
            return TC_ERR_CUDA;
        }
        TC_CUDA(cudaMalloc(&b.ws, kBlasWorkspace));
    }
    // setting the stream resets the workspace: set both every time
    if (cublasSetStream(b.h, s) != CUBLAS_STATUS_SUCCESS) return TC_ERR_CUDA;
    if (cublasSetWorkspace(b.h, b.ws, kBlasWorkspace) != CUBLAS_STATUS_SUCCESS) return TC_ERR_CUDA;
    *out = b.h;
    return TC_OK;
}

// The masked pass reads M only at (j, i) with j > i in column-major order
// (core edge i < j), so M is computed by blocks: with C split into B blocks
// of bs, the B(B+1)/2 blocks (R, K) with R >= K, each A_c[R, :]·A_c[:, K]
// (one batched call).  B = 1 is the whole product.
int core_blocks(int64_t C) { return (C >= 2048 && C % 8 == 0) ? 8 : 1; }

__global__ void k_core_ptrs(const uint16_t* A, float* M, int64_t C, int B, const void** pa, const void** pb,
                            void** pm) {
    const int64_t bs = C / B;
    int q = 0;
    for (int K = 0; K < B; ++K)
        for (int R = K; R < B; ++R, ++q)
            if (q == (int)threadIdx.x) {
                pa[q] = A + R * bs;              // rows R of A_c (column-major, leading dimension C)
                pb[q] = A + K * bs * C;          // columns K
                pm[q] = M + K * bs * C + R * bs; // block (R, K) of M
            }
}

cudaError_t core_gemm(cublasHandle_t h, int64_t C, const uint16_t* A, float* M, const void** pa, const void** pb,
                      void** pm) {
    const float one = 1.0f, zero = 0.0f;
    const int c = (int)C, B = core_blocks(C);
    cublasStatus_t st;
    if (B == 1) {
        // A_c is symmetric, so storage order does not matter: M = A_c · A_c
        st = cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, c, c, c, &one, A, CUDA_R_16BF, c, A, CUDA_R_16BF, c, &zero,
                          M, CUDA_R_32F, c, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    } else {
        const int bs = c / B;
        st = cublasGemmBatchedEx(h, CUBLAS_OP_N, CUBLAS_OP_N, bs, bs, c, &one, pa, CUDA_R_16BF, c, pb, CUDA_R_16BF,
                                 c, &zero, pm, CUDA_R_32F, c, B * (B + 1) / 2, CUBLAS_COMPUTE_32F,
                                 CUBLAS_GEMM_DEFAULT);
    }
    return st == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace

double core_flop(int64_t C) {
    const int B = core_blocks(C);
    return 2.0 * (double)C * C * C * (B * (B + 1) / 2) / ((double)B * B);
}

tc_status core_setup(tc_graph* g, const int32_t* dh, uint32_t flags, cudaStream_t s) {
    g->core_c = 0;
    const long long mode = g_core_mode.load();
    const int64_t n = g->n;
    if (mode == 0 || (flags & TC_BUILD_NO_CORE) || n < 3 || g->m == 0) return TC_OK;
    int64_t C = 0;
    if (mode > 0) {
        C = std::min<int64_t>((int64_t)mode, n);
    } else {
        const int64_t top = std::min<int64_t>(n, kCoreMax);
        std::vector<int32_t> h(top);
        TC_CUDA(cudaMemcpyAsync(h.data(), dh + (n - top), top * 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        double best = kMinGainMs;
        for (int c : kCoreSizes) {
            if (c > n) break;
            double wedges = 0;   // Σ C(d_H, 2) over the top c ranks: ids the core's rows stream
            for (int64_t i = top - c; i < top; ++i) wedges += 0.5 * (double)h[i] * (double)(h[i] - 1);
            const double cost = core_flop(c) / kGemmFlopPerMs + 8.0 * (double)c * c / kPassBytesPerMs;
            const double gain = wedges / kStreamIdsPerMs - cost;
            if (gain > best) {
                best = gain;
                C = c;
            }
        }
    }
    if (C >= 3) g->core_c = C;
    return TC_OK;
}

tc_status run_core(tc_graph* g, cudaStream_t s, bool edge_counts) {
    const int64_t C = g->core_c, t = g->n - C;
    if (C <= 0) return TC_OK;
    uint16_t* A = nullptr;
    float* M = nullptr;
    ull* S = nullptr;
    void** P = nullptr;   // the batched call's pointer arrays (A rows, A columns, M blocks)
    const int B = core_blocks(C), nb = B * (B + 1) / 2;
    TC_TRY(dalloc((void**)&A, (size_t)C * C * 2, s));
    tc_status st = dalloc((void**)&M, (size_t)C * C * 4, s);
    if (st == TC_OK) st = dalloc((void**)&S, (size_t)(C + 1) * 8, s);
    if (st == TC_OK) st = dalloc((void**)&P, (size_t)3 * nb * sizeof(void*), s);
    if (st == TC_OK) {
        st = [&]() -> tc_status {
            TC_CUDA(cudaMemsetAsync(A, 0, (size_t)C * C * 2, s));
            TC_CUDA(cudaMemsetAsync(S, 0, (size_t)(C + 1) * 8, s));
            {
                launch_scope ls("count_core_fill", s);
                k_core_fill<<<warp_blocks(C), kCoreThreads, 0, s>>>(g->row_ptr, g->hstart, g->col, t, C, A);
                TC_LAUNCH_CHECK();
            }
            const void** pa = (const void**)P;
            const void** pb = (const void**)(P + nb);
            void** pm = P + 2 * nb;
            if (B > 1) {
                launch_scope ls("count_core_ptrs", s);
                k_core_ptrs<<<1, nb, 0, s>>>(A, M, C, B, pa, pb, pm);
                TC_LAUNCH_CHECK();
            }
            cublasHandle_t h = nullptr;
            TC_TRY(blas_on(s, &h));
            {
                launch_scope ls("count_core_gemm", s);
                const int64_t k = library_kernels("core_gemm", C, B, [&](cudaStream_t p) {
                    cublasHandle_t hp = nullptr;
                    if (blas_on(p, &hp) != TC_OK) return cudaErrorUnknown;
                    return core_gemm(hp, C, A, M, pa, pb, pm);
                });
                TC_TRY(blas_on(s, &h));
                TC_CUDA(core_gemm(h, C, A, M, pa, pb, pm));
                add_launches(k - 1);
            }
            {
                launch_scope ls("count_core_edges", s);
                k_core_edges<<<warp_blocks(C), kCoreThreads, 0, s>>>(g->row_ptr, g->hstart, g->col, t, C, M, S,
                                                                     g->flag, edge_counts ? g->ecnt : nullptr,
                                                                     S + C);
                TC_LAUNCH_CHECK();
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
    if (P) dfree(P, s);
    if (S) dfree(S, s);
    if (M) dfree(M, s);
    dfree(A, s);
    return st;
}

}  // namespace tcx

extern "C" tc_status tc_set_dense_core(long long c) {
    if (c < -1) return TC_ERR_INVALID_ARG;
    tcx::g_core_mode.store(c);
    return TC_OK;
}
