// Serving: a request loop over the batch path.
//
// Callers submit graphs (host pair lists) at any time.  Worker threads, each
// with its own stream, take the requests waiting in arrival order and run as
// many of them together as fit — one batch per turn, up to an edge cap and
// within the device-memory budget left by the batches already in flight —
// so requests that arrive while others are on the GPU join the next batch
// (continuous batching), and with two workers one batch's packing, copy and
// build overlap another's count and gather on the device.  A request whose
// own estimate exceeds the whole budget is refused at submission without
// touching the device.  Results land in the caller's host buffers; each
// request records its submission, start and completion times.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tc_internal.cuh"

namespace {

using clock_t_ = std::chrono::steady_clock;

struct request {
    int64_t id;
    const int32_t* src;
    const int32_t* dst;
    int64_t np, n;
    uint64_t* out_tri;
    double* out_tc;
    int64_t bytes;
    tc_request_info info;
};

}  // namespace

struct tc_server {
    int device = 0;
    int64_t budget = 0, max_batch_pairs = 0;
    clock_t_::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<request*> pending;
    std::vector<request*> done;
    int64_t in_use = 0, next_id = 0, batches = 0, running = 0;
    bool stop = false;
    std::vector<std::thread> workers;

    double now() const { return std::chrono::duration<double>(clock_t_::now() - t0).count(); }
};

namespace {

// Device bytes a request may hold at the peak of its build (pair copies and
// sort buffers per pair, CSR and workspace per edge and vertex), rounded up.
int64_t estimate_bytes(int64_t np, int64_t n) { return 176 * np + 160 * n + (16ll << 20); }

// Requests below this many pairs are packed through pinned host staging
// (one copy each way for all of them); larger ones move directly between
// the caller's memory and the device.
constexpr int64_t kDirectPairs = 1 << 18;

struct pinned {
    void* p = nullptr;
    int64_t cap = 0;
    bool reserve(int64_t bytes) {
        if (bytes <= cap) return true;
        cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        if (cudaMallocHost(&p, bytes * 2) != cudaSuccess) return false;
        cap = bytes * 2;
        return true;
    }
    void release() {
        cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

struct staging {
    pinned pairs, results;
    void release() {
        pairs.release();
        results.release();
    }
};

// Runs one batch of requests as a disjoint union on stream s and fills each
// request's results.  Small requests come first in the union so that their
// pairs and results travel as one staged block.
tc_status run_requests(std::vector<request*>& batch, staging& stg, cudaStream_t s) {
    std::stable_partition(batch.begin(), batch.end(), [](const request* r) { return r->np < kDirectPairs; });
    const int64_t G = (int64_t)batch.size();
    std::vector<int64_t> poff(G + 1, 0), voff(G + 1, 0), nv(G, 0);
    int64_t small = 0, small_pairs = 0, small_n = 0;
    for (int64_t k = 0; k < G; ++k) {
        poff[k + 1] = poff[k] + batch[k]->np;
        voff[k + 1] = voff[k] + batch[k]->n;
        nv[k] = batch[k]->n;
        if (batch[k]->np < kDirectPairs) {
            small = k + 1;
            small_pairs = poff[k + 1];
            small_n = voff[k + 1];
        }
    }
    const int64_t np = poff[G], n = voff[G];
    if (!stg.pairs.reserve(std::max<int64_t>(small_pairs, 1) * 8) ||
        !stg.results.reserve(std::max<int64_t>(small_n * 16 + G * 8, 16)))
        return TC_ERR_OUT_OF_MEMORY;
    int32_t* hs = (int32_t*)stg.pairs.p;
    int32_t* hd = hs + small_pairs;
    for (int64_t k = 0; k < small; ++k) {
        if (batch[k]->np == 0) continue;
        std::memcpy(hs + poff[k], batch[k]->src, batch[k]->np * 4);
        std::memcpy(hd + poff[k], batch[k]->dst, batch[k]->np * 4);
    }
    int32_t* d_pairs = nullptr;
    uint64_t *d_tri = nullptr, *d_tot = nullptr;
    double* d_tc = nullptr;
    tc_batch* b = nullptr;
    tc_status st = tcx::dalloc((void**)&d_pairs, (2 * np + 1) * 4, s);
    auto H2D = [&](void* dst, const void* src, int64_t bytes) {
        if (st >= 0 && bytes > 0)
            st = tcx::from_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    };
    auto D2H = [&](void* dst, const void* src, int64_t bytes) {
        if (st >= 0 && bytes > 0)
            st = tcx::from_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    };
    int32_t* d_src = d_pairs;
    int32_t* d_dst = d_pairs + np;
    H2D(d_src, hs, small_pairs * 4);
    H2D(d_dst, hd, small_pairs * 4);
    for (int64_t k = small; k < G; ++k) {
        H2D(d_src + poff[k], batch[k]->src, batch[k]->np * 4);
        H2D(d_dst + poff[k], batch[k]->dst, batch[k]->np * 4);
    }
    if (st >= 0)
        st = tc_batch_build(d_src, d_dst, poff.data(), nv.data(), G, TC_IDS_INT32 | TC_IN_DEVICE, (tc_stream)s, &b);
    tcx::dfree(d_pairs, s);   // the build keeps its own copy
    std::vector<int64_t> eoff(G + 1, 0);
    if (st >= 0) st = tc_batch_info(b, nullptr, nullptr, nullptr, nullptr, eoff.data());
    if (st >= 0) st = tcx::dalloc((void**)&d_tri, (n + 1) * 8, s);
    if (st >= 0) st = tcx::dalloc((void**)&d_tc, (n + 1) * 8, s);
    if (st >= 0) st = tcx::dalloc((void**)&d_tot, (G + 1) * 8, s);
    if (st >= 0) st = tc_batch_run(b, d_tri, nullptr, nullptr, d_tc, d_tot, (tc_stream)s);
    uint64_t* h_tri = (uint64_t*)stg.results.p;
    double* h_tc = (double*)(h_tri + small_n);
    uint64_t* h_tot = (uint64_t*)(h_tc + small_n);
    D2H(h_tri, d_tri, small_n * 8);
    D2H(h_tc, d_tc, small_n * 8);
    D2H(h_tot, d_tot, G * 8);
    for (int64_t k = small; k < G; ++k) {
        if (batch[k]->out_tri) D2H(batch[k]->out_tri, d_tri + voff[k], batch[k]->n * 8);
        if (batch[k]->out_tc) D2H(batch[k]->out_tc, d_tc + voff[k], batch[k]->n * 8);
    }
    if (st >= 0) st = tcx::from_cuda(cudaStreamSynchronize(s));
    tcx::dfree(d_tri, s);
    tcx::dfree(d_tc, s);
    tcx::dfree(d_tot, s);
    if (b) tc_batch_free(b);
    if (st < 0) return st;
    for (int64_t k = 0; k < G; ++k) {
        request* r = batch[k];
        if (k < small) {
            if (r->out_tri) std::memcpy(r->out_tri, h_tri + voff[k], r->n * 8);
            if (r->out_tc) std::memcpy(r->out_tc, h_tc + voff[k], r->n * 8);
        }
        r->info.triangles = h_tot[k];
        r->info.edges = eoff[k + 1] - eoff[k];
        r->info.status = h_tot[k] == 0 ? TC_NO_TRIANGLES : TC_OK;
    }
    return TC_OK;
}

void worker_main(tc_server* srv) {
    cudaSetDevice(srv->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    staging stg;
    for (;;) {
        std::vector<request*> batch;
        int64_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            // wait for work whose head fits in the memory left
            srv->cv_work.wait(lk, [&] {
                return srv->stop || (!srv->pending.empty() &&
                                     srv->in_use + srv->pending.front()->bytes <= srv->budget);
            });
            if (srv->stop) break;
            int64_t edges = 0;
            while (!srv->pending.empty()) {
                request* r = srv->pending.front();
                const bool first = batch.empty();
                if (!first && (edges + r->np > srv->max_batch_pairs ||
                               srv->in_use + bytes + r->bytes > srv->budget))
                    break;
                srv->pending.pop_front();
                batch.push_back(r);
                edges += r->np;
                bytes += r->bytes;
            }
            srv->in_use += bytes;
            srv->running += (int64_t)batch.size();
            srv->batches += 1;
        }
        const double t_start = srv->now();
        for (request* r : batch) r->info.t_start = t_start;
        tc_status st;
        {
            tcx::nvtx_range nr("tc_server_batch");
            st = run_requests(batch, stg, s);
        }
        if (st < 0 && batch.size() > 1) {
            // one bad request must not fail its batch-mates: rerun each alone
            for (request* r : batch) {
                std::vector<request*> one{r};
                const tc_status sr = run_requests(one, stg, s);
                if (sr < 0) r->info.status = sr;
            }
            st = TC_OK;
        }
        const double t_done = srv->now();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            for (request* r : batch) {
                if (st < 0) r->info.status = st;
                r->info.t_done = t_done;
                r->info.batch_size = (int32_t)batch.size();
                srv->done.push_back(r);
            }
            srv->in_use -= bytes;
            srv->running -= (int64_t)batch.size();
        }
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
    stg.release();
    cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

tc_status tc_server_create(int64_t memory_budget_bytes, int64_t max_batch_pairs, int workers,
                           tc_server** out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    if (memory_budget_bytes <= 0 || max_batch_pairs <= 0 || workers < 1 || workers > 8)
        return TC_ERR_INVALID_ARG;
    tc_server* srv = new (std::nothrow) tc_server();
    if (!srv) return TC_ERR_OUT_OF_MEMORY;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return TC_ERR_CUDA;
    }
    srv->budget = memory_budget_bytes;
    srv->max_batch_pairs = max_batch_pairs;
    srv->t0 = clock_t_::now();
    try {
        for (int i = 0; i < workers; ++i) srv->workers.emplace_back(worker_main, srv);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->stop = true;
        }
        srv->cv_work.notify_all();
        for (auto& t : srv->workers) t.join();
        delete srv;
        return TC_ERR_OUT_OF_MEMORY;
    }
    *out = srv;
    return TC_OK;
}

tc_status tc_server_submit(tc_server* srv, const int32_t* h_src, const int32_t* h_dst, int64_t num_pairs,
                           int64_t n, uint64_t* h_tri, double* h_tc, int64_t* request_id) {
    if (!srv || !request_id || num_pairs < 0 || n < 0 || n > INT32_MAX ||
        (num_pairs > 0 && (!h_src || !h_dst)))
        return TC_ERR_INVALID_ARG;
    const int64_t bytes = estimate_bytes(num_pairs, n);
    if (bytes > srv->budget) return TC_ERR_OUT_OF_MEMORY;   // refused before any device work
    request* r = new (std::nothrow) request();
    if (!r) return TC_ERR_OUT_OF_MEMORY;
    r->src = h_src;
    r->dst = h_dst;
    r->np = num_pairs;
    r->n = n;
    r->out_tri = h_tri;
    r->out_tc = h_tc;
    r->bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) {
            delete r;
            return TC_ERR_STATE;
        }
        r->id = srv->next_id++;
        r->info.id = r->id;
        r->info.t_submit = srv->now();
        srv->pending.push_back(r);
    }
    *request_id = r->id;
    srv->cv_work.notify_one();
    return TC_OK;
}

tc_status tc_server_poll(tc_server* srv, tc_request_info* out, int cap, int* count, int wait_ms) {
    if (!srv || !count || cap < 0 || (cap > 0 && !out)) return TC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->done.empty() && wait_ms > 0)
        srv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !srv->done.empty(); });
    int k = 0;
    while (k < cap && !srv->done.empty()) {
        request* r = srv->done.back();
        srv->done.pop_back();
        out[k++] = r->info;
        delete r;
    }
    *count = k;
    return TC_OK;
}

tc_status tc_server_stats(tc_server* srv, int64_t* batches, int64_t* waiting, int64_t* running,
                          int64_t* memory_in_use) {
    if (!srv) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (batches) *batches = srv->batches;
    if (waiting) *waiting = (int64_t)srv->pending.size();
    if (running) *running = srv->running;
    if (memory_in_use) *memory_in_use = srv->in_use;
    return TC_OK;
}

void tc_server_free(tc_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;   // running batches finish; waiting requests are dropped
        for (request* r : srv->pending) delete r;
        srv->pending.clear();
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers) t.join();
    for (request* r : srv->done) delete r;
    delete srv;
}

}  // extern "C"
