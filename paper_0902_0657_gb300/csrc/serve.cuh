// Serving: continuous batching of frames that arrive one at a time, of
// several code lengths, with admission by device-memory bytes. Included at
// the end of lpdec.cu (it shares the decoder's kernels and layout code).
//
// One persistent kernel (k_serve) runs while work is queued. Its CTAs take
// frames from a queue that the host appends to while the kernel runs:
//   - a frame is admitted when its region (LLRs in, results out) fits the
//     device arena, a byte budget the server fixes at creation; its LLRs are
//     copied into the region before it is queued;
//   - the queue (code index and region offset per entry) and its tail live
//     in mapped pinned host memory: the host writes an entry, then releases
//     the tail; a CTA claims the next entry with a compare-and-swap on a
//     device counter (head < tail) and acquires the tail before reading it;
//   - a CTA copies the frame's LLRs into its own scratch past L1 (regions are
//     reused), decodes the frame with the same device code as the batch
//     entry points (so a result is the same alone and in the mix), writes
//     the results into the region, and publishes completion in a mapped
//     done flag after a system-scope fence;
//   - a frame cancelled while it runs stops at its next check of the entry's
//     cancel flag (between LPs, every fourth interior-point iteration);
//   - a CTA that finds the queue empty waits, sleeping between looks, for at
//     most idle_us of device time and then exits, so the kernel ends when the
//     traffic stops; a host worker relaunches it when entries are waiting and
//     no kernel runs, copies finished results back and frees their regions.
// Every wait is bounded: a stop flag (set on destroy) and the idle limit end
// the kernel.

namespace {

struct QEntry {
    int32_t code;      // index into the server's code table
    int32_t cancel;    // 1: skip the frame (cancelled before it ran)
    long long off;     // byte offset of the frame's region in the arena
};

// Byte offsets inside a frame's region for a code with n bits and m checks.
struct Region {
    size_t gam, u, hard, mask, cert, stats, bytes;
};
__host__ __device__ inline size_t up16(size_t v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline Region region_of(int n, int m) {
    Region r;
    r.gam = 0;
    r.u = up16(r.gam + 8 * (size_t)n);
    r.hard = up16(r.u + 8 * (size_t)n);
    r.mask = up16(r.hard + (size_t)n);
    r.cert = up16(r.mask + 4 * (size_t)m);
    r.stats = up16(r.cert + 4);
    r.bytes = (r.stats + sizeof(lpdec_stats) + 255) / 256 * 256;
    return r;
}

__device__ __forceinline__ uint32_t ld_acquire_sys(const volatile uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename T>
__global__ void __launch_bounds__(512)
k_serve(const CodeView* __restrict__ codes, DevParams P, Layout L, Layout Lw, char* arena,
        const volatile QEntry* q, const volatile uint32_t* tail, uint32_t* head,
        volatile uint32_t* done, const volatile uint32_t* stop, uint32_t qmask, long long idle_ns,
        char* gscratch) {
    KERNEL_PROLOGUE
    char* gw = gscratch + (size_t)blockIdx.x * L.stride + L.gbytes;
    const Layout* lw = Lw.gbytes ? &Lw : nullptr;
    int bound = -1;
    CodeView C{};
    for (;;) {
        if (B.tid == 0) {
            long long f = -1;
            const unsigned long long t0 = global_ns();
            for (long long spin = 0; spin < (1LL << 24); ++spin) {   // and by idle_ns
                if (*stop) break;
                const uint32_t t = ld_acquire_sys(tail);
                const uint32_t h = *(volatile uint32_t*)head;
                if (h < t) {
                    if (atomicCAS(head, h, h + 1) == h) { f = h; break; }
                    continue;
                }
                if ((long long)(global_ns() - t0) > idle_ns) break;
                __nanosleep(2000);
            }
            ks.next = (int)f;
            if (f >= 0) {   // one read of the entry for the whole CTA
                const uint32_t sl = (uint32_t)f & qmask;
                ks.qcode = q[sl].code;
                ks.qcancel = q[sl].cancel;
                ks.qoff = q[sl].off;
            }
        }
        __syncthreads();
        const int f = ks.next;
        const int ci = ks.qcode;
        const bool cancelled = ks.qcancel != 0;
        const long long off = ks.qoff;
        __syncthreads();
        if (f < 0) break;
        const uint32_t slot = (uint32_t)f & qmask;
        if (!cancelled) {
            if (ci != bound) {
                CodeView cv;
                const int* src = reinterpret_cast<const int*>(codes + ci);
                int* dst = reinterpret_cast<int*>(&cv);
                for (int k = 0; k < (int)(sizeof(CodeView) / sizeof(int)); ++k) dst[k] = __ldcg(src + k);
                C = bind_code<T>(cv, W);
                bound = ci;
            }
            const Region rg = region_of(C.n, C.m);
            char* base = arena + off;
            const double* g_src = reinterpret_cast<const double*>(base + rg.gam);
            for (int i = B.tid; i < C.n; i += B.nt) W.gam[i] = __ldcg(g_src + i);
            __syncthreads();
            FrameOut o{reinterpret_cast<double*>(base + rg.u),
                       reinterpret_cast<uint8_t*>(base + rg.hard),
                       reinterpret_cast<int32_t*>(base + rg.cert),
                       reinterpret_cast<uint32_t*>(base + rg.mask),
                       reinterpret_cast<lpdec_stats*>(base + rg.stats)};
            DevParams Pf = P;   // lpdec_cancel stops the frame while it runs
            Pf.abort = &q[slot].cancel;
            decode_frame<T>(B, C, W, Pf, W.gam, o, 0, ks.shscan, lw, gw);
        }
        __syncthreads();
        if (B.tid == 0) {
            __threadfence_system();
            done[slot] = (uint32_t)f + 1u;
        }
    }
}

// First-fit allocator of byte ranges of the arena (host side).
struct Arena {
    std::map<size_t, size_t> free_;   // offset -> size
    size_t used = 0;
    void init(size_t bytes) { free_.clear(); free_[0] = bytes; used = 0; }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used += bytes;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Ticket {
    uint32_t qi;         // queue index (publication order)
    int code;            // index into the code table
    size_t off, bytes;   // region
    int state;           // 0 queued/running, 1 done (results held), 2 cancelled
    double* h_res;       // results copied back (u, hard, mask, cert, stats as in the region)
};

}  // namespace

struct lpdec_server {
    int device = 0;
    lpdec_params prm{};
    lpdec_ctx* ctx = nullptr;              // plan and scratch
    std::vector<const lpdec_code*> codes;
    CodeView* d_codes = nullptr;
    Launch ln{};
    bool mixed = false;
    char* arena = nullptr;
    Arena alloc;
    uint32_t qsize = 0, qmask = 0;
    QEntry* h_q = nullptr;                 // mapped
    uint32_t* h_tail = nullptr;            // mapped: [0] tail, [1] stop
    uint32_t* h_done = nullptr;            // mapped
    QEntry* d_q = nullptr;
    uint32_t *d_tail = nullptr, *d_stop = nullptr, *d_done = nullptr;
    uint32_t* d_head = nullptr;
    cudaStream_t ks = nullptr, cs = nullptr, us = nullptr;
    cudaEvent_t kdone = nullptr;
    bool running = false;
    uint32_t published = 0;
    long long idle_ns = 2000000;
    std::map<uint64_t, Ticket> tickets;
    std::map<uint32_t, uint64_t> inflight;   // queue index -> ticket
    uint64_t next_ticket = 0;
    int32_t error = LPDEC_OK;
    bool quit = false;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    size_t hbm_total = 0;
    size_t arena_bytes = 0;
};

namespace {

#define SCK(call)                                                               \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            snprintf(g_err, sizeof g_err, "%s: %s", #call, cudaGetErrorString(e_)); \
            return LPDEC_ERR_CUDA;                                              \
        }                                                                       \
    } while (0)

int32_t serve_launch(lpdec_server* s) {
    const DevParams dp = to_dev(s->prm);
    if (s->mixed)
        k_serve<float><<<s->ln.grid, s->ln.threads, s->ln.L.smem_bytes, s->ks>>>(
            s->d_codes, dp, s->ln.L, s->ln.Lw, s->arena, s->d_q, s->d_tail, s->d_head, s->d_done,
            s->d_stop, s->qmask, s->idle_ns, s->ctx->gscratch);
    else
        k_serve<double><<<s->ln.grid, s->ln.threads, s->ln.L.smem_bytes, s->ks>>>(
            s->d_codes, dp, s->ln.L, s->ln.Lw, s->arena, s->d_q, s->d_tail, s->d_head, s->d_done,
            s->d_stop, s->qmask, s->idle_ns, s->ctx->gscratch);
    SCK(cudaGetLastError());
    SCK(cudaEventRecord(s->kdone, s->ks));
    s->running = true;
    return LPDEC_OK;
}

// Copies a finished frame's results out of its region and frees it (lock held).
int32_t serve_harvest(lpdec_server* s, Ticket& t) {
    const lpdec_code* c = s->codes[t.code];
    const Region rg = region_of(c->n, c->m);
    SCK(cudaMemcpyAsync(t.h_res, s->arena + t.off + rg.u, rg.bytes - rg.u, cudaMemcpyDeviceToHost,
                        s->cs));
    SCK(cudaStreamSynchronize(s->cs));
    s->alloc.release(t.off, t.bytes);
    t.state = t.state == 2 ? 3 : 1;   // a cancelled frame is dropped by the caller below
    return LPDEC_OK;
}

void serve_worker(lpdec_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->quit) {
        // finished frames
        bool any = false;
        for (auto it = s->inflight.begin(); it != s->inflight.end();) {
            const uint32_t qi = it->first;
            const uint32_t v = __atomic_load_n(&s->h_done[qi & s->qmask], __ATOMIC_ACQUIRE);
            if (v == qi + 1u) {
                Ticket& t = s->tickets[it->second];
                int32_t rc = serve_harvest(s, t);
                if (rc && !s->error) s->error = rc;
                if (t.state == 3) {
                    std::free(t.h_res);
                    s->tickets.erase(it->second);
                }
                it = s->inflight.erase(it);
                any = true;
            } else {
                ++it;
            }
        }
        if (any) s->cv.notify_all();
        // the kernel: relaunch while entries wait and none runs
        if (s->running && cudaEventQuery(s->kdone) == cudaSuccess) s->running = false;
        if (!s->running && !s->error) {
            uint32_t head = 0;
            if (cudaMemcpyAsync(&head, s->d_head, 4, cudaMemcpyDeviceToHost, s->cs) != cudaSuccess ||
                cudaStreamSynchronize(s->cs) != cudaSuccess) {
                s->error = LPDEC_ERR_CUDA;
            } else if (head < s->published) {
                int32_t rc = serve_launch(s);
                if (rc) s->error = rc;
            }
        }
        if (s->inflight.empty() && !s->running)
            s->cv.wait(lk, [s] { return s->quit || !s->inflight.empty(); });
        else
            s->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

void serve_free(lpdec_server* s) {
    if (s->ks) cudaStreamSynchronize(s->ks);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->ks) cudaStreamDestroy(s->ks);
    if (s->cs) cudaStreamDestroy(s->cs);
    if (s->us) cudaStreamDestroy(s->us);
    cudaFree(s->arena);
    cudaFree(s->d_codes);
    cudaFree(s->d_head);
    cudaFreeHost(s->h_q);
    cudaFreeHost(s->h_tail);
    cudaFreeHost(s->h_done);
    for (auto& kv : s->tickets) std::free(kv.second.h_res);
    if (s->ctx) lpdec_ctx_destroy(s->ctx);
    delete s;
}

}  // namespace

extern "C" {

int32_t lpdec_server_create(int32_t device, const lpdec_params* params, int32_t ncodes,
                            const lpdec_code* const* codes, size_t hbm_budget_bytes,
                            int32_t max_pending, lpdec_server** out) {
    if (!out || ncodes < 1 || !codes || max_pending < 1 || max_pending > (1 << 20))
        return LPDEC_ERR_INVALID_ARG;
    *out = nullptr;
    for (int k = 0; k < ncodes; ++k)
        if (!codes[k] || codes[k]->device != device) return LPDEC_ERR_INVALID_ARG;
    auto* s = new (std::nothrow) lpdec_server;
    if (!s) return LPDEC_ERR_INVALID_ARG;
    s->device = device;
    if (params) s->prm = *params; else lpdec_default_params(&s->prm);
    int32_t rc = lpdec_ctx_create(device, &s->prm, 0, &s->ctx);
    if (rc) { delete s; return rc; }
    s->codes.assign(codes, codes + ncodes);
    s->mixed = s->prm.precision == LPDEC_MIXED;
    // workspace for the largest code; scratch for the full grid
    Dims dims;
    std::vector<CodeView> views;
    size_t max_region = 0;
    for (const lpdec_code* c : s->codes) {
        views.push_back(view_of(c, s->prm));
        dims.cover(views.back());
        max_region = std::max(max_region, region_of(c->n, c->m).bytes);
    }
    rc = s->mixed ? plan(s->ctx, dims, 1 << 30, k_serve<float>, 4, &s->ln)
                  : plan(s->ctx, dims, 1 << 30, k_serve<double>, 8, &s->ln);
    if (rc) { serve_free(s); return rc; }
    uint32_t qs = 1;
    while (qs < (uint32_t)max_pending) qs <<= 1;
    s->qsize = qs;
    s->qmask = qs - 1;
    const size_t fixed = s->ctx->gscratch_bytes + views.size() * sizeof(CodeView) + 256;
    if (hbm_budget_bytes && hbm_budget_bytes < fixed + max_region) {
        snprintf(g_err, sizeof g_err, "HBM budget below the scratch (%zu bytes) plus one frame",
                 fixed);
        serve_free(s);
        return LPDEC_ERR_OUT_OF_BUDGET;
    }
    const size_t arena_bytes = hbm_budget_bytes ? hbm_budget_bytes - fixed
                                                : max_region * (size_t)max_pending;
    s->hbm_total = fixed + arena_bytes;
    s->arena_bytes = arena_bytes;
    bool ok = cudaMalloc(&s->arena, arena_bytes) == cudaSuccess &&
              cudaMalloc(&s->d_codes, views.size() * sizeof(CodeView)) == cudaSuccess &&
              cudaMalloc(&s->d_head, 256) == cudaSuccess &&
              cudaHostAlloc(&s->h_q, qs * sizeof(QEntry), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s->h_tail, 64, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s->h_done, qs * sizeof(uint32_t), cudaHostAllocMapped) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->ks, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->us, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        snprintf(g_err, sizeof g_err, "server allocation failed");
        serve_free(s);
        return LPDEC_ERR_CUDA;
    }
    std::memset(s->h_q, 0, qs * sizeof(QEntry));
    std::memset(s->h_tail, 0, 64);
    std::memset(s->h_done, 0, qs * sizeof(uint32_t));
    void* p = nullptr;
    ok = cudaHostGetDevicePointer(&p, s->h_q, 0) == cudaSuccess;
    s->d_q = static_cast<QEntry*>(p);
    ok = ok && cudaHostGetDevicePointer(&p, s->h_tail, 0) == cudaSuccess;
    s->d_tail = static_cast<uint32_t*>(p);
    s->d_stop = s->d_tail + 1;
    ok = ok && cudaHostGetDevicePointer(&p, s->h_done, 0) == cudaSuccess;
    s->d_done = static_cast<uint32_t*>(p);
    ok = ok && cudaMemcpy(s->d_codes, views.data(), views.size() * sizeof(CodeView),
                          cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(s->d_head, 0, 256) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        snprintf(g_err, sizeof g_err, "server set-up failed");
        serve_free(s);
        return LPDEC_ERR_CUDA;
    }
    s->alloc.init(arena_bytes);
    s->worker = std::thread(serve_worker, s);
    *out = s;
    return LPDEC_OK;
}

int32_t lpdec_submit(lpdec_server* s, const lpdec_code* code, const double* gamma,
                     uint64_t* ticket) {
    if (!s || !code || !gamma || !ticket) return LPDEC_ERR_INVALID_ARG;
    int ci = -1;
    for (size_t k = 0; k < s->codes.size(); ++k)
        if (s->codes[k] == code) { ci = (int)k; break; }
    if (ci < 0) return LPDEC_ERR_INVALID_ARG;
    for (int i = 0; i < code->n; ++i)
        if (!std::isfinite(gamma[i])) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->error) return s->error;
    const Region rg = region_of(code->n, code->m);
    if (s->inflight.size() >= s->qsize) return LPDEC_ERR_OUT_OF_BUDGET;
    size_t off = 0;
    if (!s->alloc.alloc(rg.bytes, &off)) return LPDEC_ERR_OUT_OF_BUDGET;
    double* res = static_cast<double*>(std::malloc(rg.bytes));
    if (!res) { s->alloc.release(off, rg.bytes); return LPDEC_ERR_INVALID_ARG; }
    if (cudaSetDevice(s->device) != cudaSuccess ||
        cudaMemcpyAsync(s->arena + off + rg.gam, gamma, 8 * (size_t)code->n,
                        cudaMemcpyHostToDevice, s->us) != cudaSuccess ||
        cudaStreamSynchronize(s->us) != cudaSuccess) {
        std::free(res);
        s->alloc.release(off, rg.bytes);
        s->error = LPDEC_ERR_CUDA;
        return LPDEC_ERR_CUDA;
    }
    const uint32_t qi = s->published;
    QEntry& e = s->h_q[qi & s->qmask];
    e.code = ci;
    e.cancel = 0;
    e.off = (long long)off;
    __atomic_store_n(&s->h_tail[0], qi + 1u, __ATOMIC_RELEASE);   // publish
    s->published = qi + 1u;
    *ticket = s->next_ticket++;
    s->tickets[*ticket] = Ticket{qi, ci, off, rg.bytes, 0, res};
    s->inflight[qi] = *ticket;
    s->cv.notify_all();
    return LPDEC_OK;
}

int32_t lpdec_poll(lpdec_server* s, uint64_t ticket, double* u_out, uint8_t* hard_out,
                   int32_t* cert_out, uint32_t* cut_mask_out, lpdec_stats* stats) {
    if (!s) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end() || it->second.state >= 2) return LPDEC_ERR_INVALID_ARG;
    if (it->second.state == 0) return s->error ? s->error : LPDEC_ERR_PENDING;
    const Ticket& t = it->second;
    const lpdec_code* c = s->codes[t.code];
    const Region rg = region_of(c->n, c->m);
    const char* h = reinterpret_cast<const char*>(t.h_res);   // the region from rg.u on
    if (u_out) std::memcpy(u_out, h, 8 * (size_t)c->n);
    if (hard_out) std::memcpy(hard_out, h + (rg.hard - rg.u), (size_t)c->n);
    if (cut_mask_out) std::memcpy(cut_mask_out, h + (rg.mask - rg.u), 4 * (size_t)c->m);
    if (cert_out) std::memcpy(cert_out, h + (rg.cert - rg.u), 4);
    if (stats) std::memcpy(stats, h + (rg.stats - rg.u), sizeof(lpdec_stats));
    std::free(t.h_res);
    s->tickets.erase(it);
    return LPDEC_OK;
}

int32_t lpdec_cancel(lpdec_server* s, uint64_t ticket) {
    if (!s) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end() || it->second.state >= 2) return LPDEC_ERR_INVALID_ARG;
    Ticket& t = it->second;
    if (t.state == 1) {   // finished, not yet polled: release now
        std::free(t.h_res);
        s->tickets.erase(it);
        return LPDEC_OK;
    }
    // queued or running: a CTA that has not claimed it yet skips it; either
    // way its region and ticket are released when the kernel reports it done
    __atomic_store_n(&s->h_q[t.qi & s->qmask].cancel, 1, __ATOMIC_RELEASE);
    t.state = 2;
    return LPDEC_OK;
}

int32_t lpdec_server_stats(lpdec_server* s, size_t* hbm_bytes, size_t* arena_bytes,
                           size_t* arena_used, int32_t* outstanding) {
    if (!s) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (hbm_bytes) *hbm_bytes = s->hbm_total;
    if (arena_bytes) *arena_bytes = s->arena_bytes;
    if (arena_used) *arena_used = s->alloc.used;
    if (outstanding) *outstanding = (int32_t)s->tickets.size();
    return LPDEC_OK;
}

int32_t lpdec_server_destroy(lpdec_server* s) {
    if (!s) return LPDEC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->quit = true;
        __atomic_store_n(&s->h_tail[1], 1u, __ATOMIC_RELEASE);   // stop the kernel's waits
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    serve_free(s);
    return LPDEC_OK;
}

}  // extern "C"
