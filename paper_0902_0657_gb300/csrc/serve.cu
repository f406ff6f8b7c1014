// Serving layer of the decoder: frames are submitted one at a time as they
// arrive and decoded in batches that overlap on the GPU (continuous batching
// at batch granularity).
//
// A server owns L lanes. Each lane is a decoder context of its own (stream,
// per-CTA scratch, copy of the code) with pinned host and device buffers for
// up to B frames. A worker thread moves frames from the queue of submitted
// requests to an idle lane, copies them in, launches the persistent decode
// kernel on the lane's stream, copies the results back and records an event.
// While one lane's batch runs out its tail of slow frames, and its CTAs
// leave SMs idle one by one, the next lane's batch is launched on another
// stream and takes those SMs, so requests that arrive while others are on
// the GPU are admitted as lanes free up. A frame's result never depends on
// the other frames of its batch (one CTA decodes one frame from start to
// end), so a result is the same alone and in the mix.
//
// Admission: at most max_pending requests may be queued or in flight;
// lpdec_submit returns LPDEC_ERR_OUT_OF_BUDGET beyond that.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lpdec.h"

namespace {

struct Lane {
    lpdec_ctx* ctx = nullptr;
    lpdec_code* code = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    double *h_gamma = nullptr, *h_u = nullptr;
    uint8_t* h_hard = nullptr;
    int32_t* h_cert = nullptr;
    lpdec_stats* h_stats = nullptr;
    double *d_gamma = nullptr, *d_u = nullptr;
    uint8_t* d_hard = nullptr;
    int32_t* d_cert = nullptr;
    lpdec_stats* d_stats = nullptr;
    std::vector<uint64_t> tickets;   // frames of the batch in flight (empty = idle)
};

struct Result {
    std::vector<double> u;
    std::vector<uint8_t> hard;
    int32_t cert = 0;
    lpdec_stats stats{};
};

}  // namespace

struct lpdec_server {
    int device = 0;
    int n = 0, m = 0;
    int batch = 0;
    int max_pending = 0;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::pair<uint64_t, std::vector<double>>> queue;
    std::unordered_map<uint64_t, Result> results;
    std::unordered_set<uint64_t> live;   // issued and not yet polled
    uint64_t next_ticket = 0;
    int outstanding = 0;    // queued + in flight + finished but not polled
    int32_t error = LPDEC_OK;
    bool stop = false;
    std::thread worker;
};

namespace {

void free_lane(Lane& l) {
    if (l.stream) cudaStreamSynchronize(l.stream);
    if (l.done) cudaEventDestroy(l.done);
    if (l.stream) cudaStreamDestroy(l.stream);
    cudaFreeHost(l.h_gamma); cudaFreeHost(l.h_u); cudaFreeHost(l.h_hard);
    cudaFreeHost(l.h_cert); cudaFreeHost(l.h_stats);
    cudaFree(l.d_gamma); cudaFree(l.d_u); cudaFree(l.d_hard); cudaFree(l.d_cert);
    cudaFree(l.d_stats);
    if (l.code) lpdec_code_destroy(l.code);
    if (l.ctx) lpdec_ctx_destroy(l.ctx);
    l = Lane{};
}

int32_t make_lane(Lane& l, int device, const lpdec_params* prm, int m, int n,
                  const int32_t* row_ptr, const int32_t* col_idx, int B) {
    int32_t rc = lpdec_ctx_create(device, prm, 0, &l.ctx);
    if (rc) return rc;
    rc = lpdec_code_create(l.ctx, m, n, row_ptr, col_idx, &l.code);
    if (rc) return rc;
    const size_t nb = (size_t)B * n;
    bool ok = cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMallocHost(&l.h_gamma, nb * 8) == cudaSuccess &&
              cudaMallocHost(&l.h_u, nb * 8) == cudaSuccess &&
              cudaMallocHost(&l.h_hard, nb) == cudaSuccess &&
              cudaMallocHost(&l.h_cert, (size_t)B * 4) == cudaSuccess &&
              cudaMallocHost(&l.h_stats, (size_t)B * sizeof(lpdec_stats)) == cudaSuccess &&
              cudaMalloc(&l.d_gamma, nb * 8) == cudaSuccess &&
              cudaMalloc(&l.d_u, nb * 8) == cudaSuccess &&
              cudaMalloc(&l.d_hard, nb) == cudaSuccess &&
              cudaMalloc(&l.d_cert, (size_t)B * 4) == cudaSuccess &&
              cudaMalloc(&l.d_stats, (size_t)B * sizeof(lpdec_stats)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return LPDEC_ERR_CUDA;
    }
    // one frame whose hard decision is a codeword (no LP): sizes the lane's
    // scratch now, so that no allocation falls between overlapping batches
    for (int i = 0; i < n; ++i) l.h_gamma[i] = 1.0;
    if (cudaMemcpyAsync(l.d_gamma, l.h_gamma, (size_t)n * 8, cudaMemcpyHostToDevice, l.stream))
        return LPDEC_ERR_CUDA;
    rc = lpdec_decode_batch_device(l.ctx, l.code, 1, l.d_gamma, l.d_u, l.d_hard, l.d_cert,
                                   nullptr, l.d_stats, l.stream);
    if (rc) return rc;
    if (cudaStreamSynchronize(l.stream)) return LPDEC_ERR_CUDA;
    return LPDEC_OK;
}

// Copies the finished batch of lane l into the result map (lock held).
void harvest(lpdec_server* s, Lane& l) {
    const size_t n = s->n;
    for (size_t k = 0; k < l.tickets.size(); ++k) {
        Result r;
        r.u.assign(l.h_u + k * n, l.h_u + (k + 1) * n);
        r.hard.assign(l.h_hard + k * n, l.h_hard + (k + 1) * n);
        r.cert = l.h_cert[k];
        r.stats = l.h_stats[k];
        s->results.emplace(l.tickets[k], std::move(r));
    }
    l.tickets.clear();
}

// Starts a batch of up to B queued frames on idle lane l (lock held).
int32_t launch(lpdec_server* s, Lane& l) {
    const size_t n = s->n;
    const int k = (int)std::min<size_t>(s->queue.size(), (size_t)s->batch);
    for (int f = 0; f < k; ++f) {
        auto& req = s->queue.front();
        std::memcpy(l.h_gamma + (size_t)f * n, req.second.data(), n * 8);
        l.tickets.push_back(req.first);
        s->queue.pop_front();
    }
    const size_t nb = (size_t)k * n;
    if (cudaMemcpyAsync(l.d_gamma, l.h_gamma, nb * 8, cudaMemcpyHostToDevice, l.stream))
        return LPDEC_ERR_CUDA;
    int32_t rc = lpdec_decode_batch_device(l.ctx, l.code, k, l.d_gamma, l.d_u, l.d_hard,
                                           l.d_cert, nullptr, l.d_stats, l.stream);
    if (rc) return rc;
    if (cudaMemcpyAsync(l.h_u, l.d_u, nb * 8, cudaMemcpyDeviceToHost, l.stream) ||
        cudaMemcpyAsync(l.h_hard, l.d_hard, nb, cudaMemcpyDeviceToHost, l.stream) ||
        cudaMemcpyAsync(l.h_cert, l.d_cert, (size_t)k * 4, cudaMemcpyDeviceToHost, l.stream) ||
        cudaMemcpyAsync(l.h_stats, l.d_stats, (size_t)k * sizeof(lpdec_stats),
                        cudaMemcpyDeviceToHost, l.stream) ||
        cudaEventRecord(l.done, l.stream))
        return LPDEC_ERR_CUDA;
    return LPDEC_OK;
}

void worker_loop(lpdec_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool busy = false;
        for (auto& l : s->lanes) {
            if (l.tickets.empty()) continue;
            cudaError_t q = cudaEventQuery(l.done);
            if (q == cudaSuccess) {
                harvest(s, l);
                s->cv.notify_all();
            } else if (q == cudaErrorNotReady) {
                busy = true;
            } else {
                s->error = LPDEC_ERR_CUDA;
                l.tickets.clear();
            }
        }
        for (auto& l : s->lanes) {
            if (s->queue.empty() || s->error) break;
            if (!l.tickets.empty()) continue;
            int32_t rc = launch(s, l);
            if (rc) s->error = rc;
            busy = true;
        }
        if (s->stop && s->queue.empty() && !busy) break;
        if (busy)   // poll the events again soon
            s->cv.wait_for(lk, std::chrono::microseconds(200));
        else
            s->cv.wait(lk, [s] { return s->stop || !s->queue.empty(); });
    }
}

}  // namespace

extern "C" {

int32_t lpdec_server_create(int32_t device, const lpdec_params* params, int32_t m, int32_t n,
                            const int32_t* row_ptr, const int32_t* col_idx, int32_t lanes,
                            int32_t batch, int32_t max_pending, lpdec_server** out) {
    if (!out || lanes < 1 || lanes > 16 || batch < 1 || max_pending < 1) return LPDEC_ERR_INVALID_ARG;
    *out = nullptr;
    auto* s = new lpdec_server;
    s->device = device;
    s->n = n;
    s->m = m;
    s->batch = batch;
    s->max_pending = max_pending;
    s->lanes.resize(lanes);
    for (auto& l : s->lanes) {
        int32_t rc = make_lane(l, device, params, m, n, row_ptr, col_idx, batch);
        if (rc) {
            for (auto& x : s->lanes) free_lane(x);
            delete s;
            return rc;
        }
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return LPDEC_OK;
}

int32_t lpdec_submit(lpdec_server* s, const double* gamma, uint64_t* ticket) {
    if (!s || !gamma || !ticket) return LPDEC_ERR_INVALID_ARG;
    for (int i = 0; i < s->n; ++i)
        if (!std::isfinite(gamma[i])) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->error) return s->error;
    if (s->outstanding >= s->max_pending) return LPDEC_ERR_OUT_OF_BUDGET;
    *ticket = s->next_ticket++;
    s->queue.emplace_back(*ticket, std::vector<double>(gamma, gamma + s->n));
    s->live.insert(*ticket);
    s->outstanding++;
    s->cv.notify_all();
    return LPDEC_OK;
}

int32_t lpdec_poll(lpdec_server* s, uint64_t ticket, double* u_out, uint8_t* hard_out,
                   int32_t* cert_out, lpdec_stats* stats) {
    if (!s) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) {
        if (!s->live.count(ticket)) return LPDEC_ERR_INVALID_ARG;   // never issued, or polled
        return s->error ? s->error : LPDEC_ERR_PENDING;
    }
    const Result& r = it->second;
    if (u_out) std::memcpy(u_out, r.u.data(), r.u.size() * 8);
    if (hard_out) std::memcpy(hard_out, r.hard.data(), r.hard.size());
    if (cert_out) *cert_out = r.cert;
    if (stats) *stats = r.stats;
    s->results.erase(it);
    s->live.erase(ticket);
    s->outstanding--;
    return LPDEC_OK;
}

int32_t lpdec_server_destroy(lpdec_server* s) {
    if (!s) return LPDEC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->queue.clear();
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& l : s->lanes) free_lane(l);
    delete s;
    return LPDEC_OK;
}

}  // extern "C"
