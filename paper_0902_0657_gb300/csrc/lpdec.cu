// Kernels and host C ABI of the adaptive LP decoder (see include/lpdec.h).
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -shared -Xcompiler -fPIC
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lpdec_device.cuh"

using namespace lpdec;

// ---------------------------------------------------------------------------
// Kernels. All are persistent: CTAs take frames from a queue counter.
// ---------------------------------------------------------------------------
namespace {

struct KernelShared {
    double red[128];
    int shscan[40];
    int next;
    int sw;
    long long qoff;   // serving: the claimed queue entry, read once by thread 0
    int qcode, qcancel;
};

// The warp of this CTA that runs its single-warp phases. A CTA's warps take
// consecutive warp slots of its SM and a slot's sub-partition is its index
// mod 4, so warp 0 of every CTA would share one sub-partition (and its FP64
// pipe); rotating by the CTA's slot block spreads them. The choice affects
// only where the work runs, never its result.
__device__ __forceinline__ int serial_warp(int nwarps) {
    unsigned slot;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(slot));
    return (int)((slot / (unsigned)nwarps) % (unsigned)nwarps);
}

__device__ __forceinline__ int next_frame(Blk& B, int* counter, int* slot) {
    if (B.tid == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    int f = *slot;
    __syncthreads();
    return f;
}

#define KERNEL_PROLOGUE                                                         \
    extern __shared__ __align__(16) char smem[];                                \
    __shared__ KernelShared ks;                                                 \
    Blk B{(int)threadIdx.x, (int)blockDim.x, (int)(threadIdx.x & 31),          \
          (int)(threadIdx.x >> 5), (int)(blockDim.x >> 5), ks.red, 0, 0};       \
    if (threadIdx.x == 0) ks.sw = serial_warp(B.nwarps);                        \
    __syncthreads();                                                            \
    B.sw = ks.sw;                                                               \
    WS<T> W = make_ws<T>(L, smem, gscratch + (size_t)blockIdx.x * L.stride);            \
    W.lanes = P.lane_policy;

// Where frame f of a batch lives: its code (index into the batch's code
// table) and the offsets of its bits and checks in the packed (ragged)
// frame-major arrays.
struct FrameDesc {
    int32_t code;
    int32_t pad;
    long long on, om;
};

// Frame order of a batch (lpdec_params.order_frames): frames expected to
// need the most LPs go first, so that the slow ones do not start last and
// leave the other CTAs idle at the end of a launch. The expectation is the
// total reliability of the hard decision's errors, sum over gamma_i < 0 of
// -gamma_i (correlation 0.56-0.64 with the number of LPs on the n = 1008
// workload at 1.5-2.5 dB). Key = complemented top bits of that sum | frame
// index (24 bits), sorted ascending: the largest sums first, ties by index.
constexpr unsigned long long kOrderIdx = (1ull << 24) - 1;

__global__ void k_order_keys(const double* __restrict__ gamma, int n, int nframes, int n2,
                             unsigned long long* keys) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int f = w; f < n2; f += nw) {
        double s = 0.0;
        if (f < nframes)
            for (int i = lane; i < n; i += 32) {
                const double g = gamma[(size_t)f * n + i];
                s += g < 0.0 ? -g : 0.0;
            }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0)
            keys[f] = f < nframes
                ? ((~((unsigned long long)__double_as_longlong(s) >> 24)) << 24) | (unsigned long long)f
                : ~0ull;
    }
}

// Bitonic sort of n2 (a power of two) keys in global memory by one CTA.
__global__ void k_sort_keys(unsigned long long* key, int n2) {
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (n2 >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (j - 1));
                const int l = i + j;
                const bool up = (i & k) == 0;
                const unsigned long long ki = key[i], kl = key[l];
                if ((ki > kl) == up) { key[i] = kl; key[l] = ki; }
            }
            __syncthreads();
        }
}

// Whole-frame decode. One code for every frame (descs == nullptr; frame f at
// f*n / f*m), or per-frame codes from codes[descs[f].code] with ragged
// offsets.
template <typename T>
__global__ void __launch_bounds__(512)
k_decode(CodeView C0, const CodeView* __restrict__ codes, const FrameDesc* __restrict__ descs,
         DevParams P, Layout L, Layout Lw, const double* __restrict__ gamma, double* u,
         uint8_t* hard, int32_t* cert, uint32_t* mask, lpdec_stats* stats, int nframes,
         int* counter, char* gscratch, const unsigned long long* __restrict__ order) {
    KERNEL_PROLOGUE
    char* gw = gscratch + (size_t)blockIdx.x * L.stride + L.gbytes;   // wide workspace
    const Layout* lw = Lw.gbytes ? &Lw : nullptr;
    CodeView C = descs ? C0 : bind_code<T>(C0, W);
    int bound = -1;
    for (;;) {
        int f = next_frame(B, counter, &ks.next);
        if (f >= nframes) break;
        if (order) f = (int)(order[f] & kOrderIdx);   // the queue's f-th frame
        long long on = (long long)f * C0.n, om = (long long)f * C0.m;
        if (descs) {
            const FrameDesc d = descs[f];
            if (d.code != bound) { C = bind_code<T>(codes[d.code], W); bound = d.code; }
            on = d.on;
            om = d.om;
        }
        FrameOut o{u + on, hard + on, cert + f, mask ? mask + om : nullptr,
                   stats ? stats + f : nullptr};
        decode_frame<T>(B, C, W, P, gamma + on, o, 0, ks.shscan, lw, gw);
    }
}

// LP state of the step kernels: one inequality per check (in_lp, mask),
// flip bits from gamma; the next lp_build makes the cut list from it.
template <typename T>
__device__ inline void load_lp_state(Blk& B, const CodeView& C, WS<T>& W, const double* g,
                                     const uint8_t* in_lp, const uint32_t* mask) {
    for (int k = B.tid; k < (C.n + 31) / 32; k += B.nt) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            int i = k * 32 + b;
            if (i < C.n && g[i] < 0.0) bits |= 1u << b;
        }
        W.flip[k] = bits;
    }
    for (int j = B.tid; j < C.m; j += B.nt) {
        W.flags[j] = in_lp[j] ? (kInLP | kNew) : 0;
        W.mask[j] = mask[j];
    }
    for (int j = B.tid; j <= C.m; j += B.nt) W.crptr[j] = 0;
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512)
k_cut_search(CodeView C0, DevParams P, Layout L, const double* u, const uint8_t* active,
             uint8_t* in_lp, uint32_t* mask, int32_t* flag, int nframes, int* counter,
             char* gscratch) {
    KERNEL_PROLOGUE
    const CodeView C = bind_code<T>(C0, W);
    for (;;) {
        int f = next_frame(B, counter, &ks.next);
        if (f >= nframes) break;
        const size_t om = (size_t)f * C.m;
        for (int i = B.tid; i < C.n; i += B.nt) W.u[i] = u[(size_t)f * C.n + i];
        for (int j = B.tid; j < C.m; j += B.nt) {
            uint8_t fl = in_lp[om + j] ? kInLP : 0;
            if (fl && active[om + j]) fl |= kActive;
            W.flags[j] = fl;
            W.mask[j] = mask[om + j];
        }
        __syncthreads();
        if (P.variant == LPDEC_MALP_B) drop_inactive<T>(B, C, W);
        int added = cut_search<T>(B, C, W, P, P.variant == LPDEC_ALP);
        for (int j = B.tid; j < C.m; j += B.nt) {
            in_lp[om + j] = (W.flags[j] & kInLP) ? 1 : 0;
            mask[om + j] = W.mask[j];
        }
        if (B.tid == 0) flag[f] = added;
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(512)
k_mts_select(CodeView C0, DevParams P, Layout L, const double* gamma, const uint8_t* in_lp,
             const uint32_t* mask, const double* wts, int32_t* col, int32_t* row,
             int nframes, int* counter, char* gscratch) {
    KERNEL_PROLOGUE
    const CodeView C = bind_code<T>(C0, W);
    const int qm = C.n + C.m;
    for (;;) {
        int f = next_frame(B, counter, &ks.next);
        if (f >= nframes) break;
        load_lp_state<T>(B, C, W, gamma + (size_t)f * C.n, in_lp + (size_t)f * C.m,
                         mask + (size_t)f * C.m);
        Frame F{0, C.n, 0.0, 0.0, 0};
        lp_build<T>(B, C, W, F, ks.shscan, false, C.pmax, C.eamax);
        for (int i = B.tid; i < F.q; i += B.nt) W.d2[i] = wts[(size_t)f * qm + i];
        __syncthreads();
        select_mts<T>(B, C, W, F, W.d2, P.precond == LPDEC_MTS_ADAPTIVE ? LPDEC_MTS_COLUMN
                                                                          : P.precond);
        selection_order<T>(B, W, F, col + (size_t)f * C.m, row + (size_t)f * C.m, C.m);
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(512)
k_pcg(CodeView C0, DevParams P, Layout L, const double* gamma, const uint8_t* in_lp,
      const uint32_t* mask, const double* d2, const double* wv, double* dy, int32_t* iters,
      int nframes, int* counter, char* gscratch) {
    KERNEL_PROLOGUE
    const CodeView C = bind_code<T>(C0, W);
    const int qm = C.n + C.m;
    for (;;) {
        int f = next_frame(B, counter, &ks.next);
        if (f >= nframes) break;
        load_lp_state<T>(B, C, W, gamma + (size_t)f * C.n, in_lp + (size_t)f * C.m,
                         mask + (size_t)f * C.m);
        Frame F{0, C.n, 0.0, 0.0, 0};
        lp_build<T>(B, C, W, F, ks.shscan, false, C.pmax, C.eamax);
        for (int i = B.tid; i < F.q; i += B.nt) W.d2[i] = d2[(size_t)f * qm + i];
        for (int r = B.tid; r < F.p; r += B.nt) W.w[r] = wv[(size_t)f * C.m + r];
        __syncthreads();
        Levels Lv = select_mts<T>(B, C, W, F, W.d2,
                                  P.precond == LPDEC_MTS_ADAPTIVE ? LPDEC_MTS_COLUMN : P.precond);
        for (int i = B.tid; i < F.q; i += B.nt) W.d2t[i] = (T)W.d2[i];
        for (int r = B.tid; r < F.p; r += B.nt) W.invd2p[r] = (T)(1.0 / W.d2[W.pivcol[r]]);
        __syncthreads();
        bool force64 = false;
        bool force_dense = false;
        NewtonOut no = newton_solve<T>(B, C, W, F, Lv, P, P.tol_pcg, P.max_pcg, force64,
                                       force_dense);
        for (int r = B.tid; r < C.m; r += B.nt) dy[(size_t)f * C.m + r] = r < F.p ? W.dy[r] : 0.0;
        if (B.tid == 0) iters[f] = no.iters;
        __syncthreads();
    }
}

// Diagnostic PCG with the context's preconditioner (or plain CG): residual
// and coefficient history per frame (pcg_traced).
template <typename T>
__global__ void __launch_bounds__(512)
k_pcg_trace(CodeView C0, DevParams P, Layout L, const double* gamma, const uint8_t* in_lp,
            const uint32_t* mask, const double* d2, const double* wv, double* dy, int32_t* iters,
            double* hist, int max_hist, int identity, double tol, int nframes, int* counter,
            char* gscratch) {
    KERNEL_PROLOGUE
    const CodeView C = bind_code<T>(C0, W);
    const int qm = C.n + C.m;
    for (;;) {
        int f = next_frame(B, counter, &ks.next);
        if (f >= nframes) break;
        load_lp_state<T>(B, C, W, gamma + (size_t)f * C.n, in_lp + (size_t)f * C.m,
                         mask + (size_t)f * C.m);
        Frame F{0, C.n, 0.0, 0.0, 0};
        lp_build<T>(B, C, W, F, ks.shscan, false, C.pmax, C.eamax);
        for (int i = B.tid; i < F.q; i += B.nt) W.d2[i] = d2[(size_t)f * qm + i];
        for (int r = B.tid; r < F.p; r += B.nt) W.r[r] = (T)wv[(size_t)f * C.m + r];
        __syncthreads();
        Levels Lv{-1, -1};
        if (!identity)
            Lv = select_mts<T>(B, C, W, F, W.d2,
                               P.precond == LPDEC_MTS_ADAPTIVE ? LPDEC_MTS_COLUMN : P.precond);
        for (int i = B.tid; i < F.q; i += B.nt) W.d2t[i] = (T)W.d2[i];
        for (int r = B.tid; r < F.p; r += B.nt) {
            const int pc = identity ? 0 : W.pivcol[r];
            W.invd2p[r] = identity ? T(1) : (T)(1.0 / W.d2[pc]);
        }
        for (int r = B.tid; r < F.p; r += B.nt) W.r[r] = (T)wv[(size_t)f * C.m + r];
        for (int k = B.tid; k < 3 * max_hist; k += B.nt) hist[(size_t)f * 3 * max_hist + k] = 0.0;
        __syncthreads();
        int it = pcg_traced<T>(B, C, W, F, Lv, identity != 0, tol, max_hist,
                               hist + (size_t)f * 3 * max_hist);
        for (int r = B.tid; r < C.m; r += B.nt) dy[(size_t)f * C.m + r] = r < F.p ? (double)W.xs[r] : 0.0;
        if (B.tid == 0) iters[f] = it;
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(512)
k_lp_solve(CodeView C0, DevParams P, Layout L, const double* gamma, const uint8_t* in_lp,
           const uint32_t* mask, double* xo, lpdec_stats* stats, int nframes, int* counter,
           char* gscratch, double* trace, int max_trace) {
    KERNEL_PROLOGUE
    double* const W0lz = reinterpret_cast<double*>(ws_ptr(L, G_LZ, smem, gscratch + (size_t)blockIdx.x * L.stride));
    const CodeView C = bind_code<T>(C0, W);
    const int qm = C.n + C.m;
    for (;;) {
        int f = next_frame(B, counter, &ks.next);
        if (f >= nframes) break;
        const double* g = gamma + (size_t)f * C.n;
        load_lp_state<T>(B, C, W, g, in_lp + (size_t)f * C.m, mask + (size_t)f * C.m);
        Frame F{0, C.n, 0.0, 0.0, 0};
        lp_build<T>(B, C, W, F, ks.shscan, false, C.pmax, C.eamax);
        lpdec_stats st{};
        if (F.p > 0) {
            IpmOut io;
            bool solved;
            if (trace) {   // one run, traced (no refinement)
                W.lz = W0lz;
                io = ipm_solve<T>(B, C, W, F, P, g, 0, trace + (size_t)f * kTrace * max_trace,
                                  max_trace);
                W.lz = nullptr;
                int ok = io.certified || certify<T>(B, C, W, F, g);
                if (!ok) st.vertex_failures = vertex_recover<T>(B, C, W, F, g);
                solved = io.converged || ok;
            } else {
                solved = solve_lp<T>(B, C, W, F, P, g, st, io);
            }
            st.ipm_iters_total = io.iters;
            st.pcg_iters_total = io.pcg_iters;
            st.pcg_iters_fp64 = io.pcg_iters64;
            st.pcg_flops = io.flops;
            st.max_levels = io.max_levels;
            st.status = solved ? LPDEC_OK : LPDEC_ERR_NOT_CONVERGED;
        } else {
            for (int i = B.tid; i < C.n; i += B.nt) W.x[i] = 0.0;
            __syncthreads();
        }
        st.lp_rows_final = F.p;
        double obj = 0.0;
        for (int i = B.tid; i < qm; i += B.nt) {
            double v = i < F.q ? W.x[i] : 0.0;
            xo[(size_t)f * qm + i] = v;
            if (i < C.n) obj += g[i] * (flipped(W.flip, i) ? 1.0 - v : v);
        }
        obj = bsum(B, obj);
        if (B.tid == 0) { st.objective = obj; stats[f] = st; }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct lpdec_ctx {
    int device = 0;
    lpdec_params prm{};
    size_t budget = 0;
    int sm_count = 0;
    int smem_optin = 0;
    int smem_per_sm = 0;
    cudaStream_t stream = nullptr;
    char* gscratch = nullptr;
    size_t gscratch_bytes = 0;
    int* counter = nullptr;
    char* staging = nullptr;     // device buffers of the host entry points
    size_t staging_bytes = 0;
    char* h_stage = nullptr;     // pinned host buffer of the host entry points
    size_t h_stage_bytes = 0;
    char* d_meta = nullptr;      // code table and frame descriptors of a mixed batch
    char* h_meta = nullptr;      // ... and their pinned host copy
    size_t meta_bytes = 0;
    cudaEvent_t meta_done = nullptr;   // the last copy out of h_meta has run
    unsigned long long* d_order = nullptr;   // frame order keys of a batch
    size_t order_n = 0;
    std::mutex mu;
};

struct lpdec_code {
    lpdec_ctx* ctx = nullptr;
    int device = 0;
    int m = 0, n = 0, E = 0;
    int dmax = 0;   // largest check degree
    int *h_ptr = nullptr, *h_col = nullptr, *e_chk = nullptr;
    int *v_ptr = nullptr, *v_chk = nullptr, *v_eidx = nullptr;
};

namespace {

thread_local char g_err[256];

#define CK(call)                                                                \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            snprintf(g_err, sizeof g_err, "%s: %s", #call, cudaGetErrorString(e_)); \
            return LPDEC_ERR_CUDA;                                              \
        }                                                                       \
    } while (0)

DevParams to_dev(const lpdec_params& p) {
    DevParams d;
    d.sigma = p.sigma; d.eta = p.eta; d.tol_gap = p.tol_gap; d.tol_feas = p.tol_feas;
    d.tol_pcg = p.tol_pcg; d.tau_act = p.tau_act; d.tau_cut = p.tau_cut; d.tau_int = p.tau_int;
    d.pcg_gap_factor = p.pcg_gap_factor; d.tol_inner = p.tol_inner;
    d.tol_feas_loose = p.tol_feas_loose;
    d.tol_cert = p.tol_cert;
    d.tau_inc = p.tau_inc;
    d.max_alp = p.max_alp; d.max_ipm = p.max_ipm; d.max_pcg = p.max_pcg;
    d.variant = p.variant; d.precision = p.precision;
    d.precond = p.precond; d.precond_switch = p.precond_switch;
    d.warm_start = p.warm_start; d.mts_reuse = p.mts_reuse;
    d.lane_policy = p.lane_policy;
    d.dense_switch = p.dense_switch;
    d.abort = nullptr;
    return d;
}

// LP row capacity of one frame (lp_rows_cap; library choice: 2m). The main
// workspace holds min(m, cap) rows, enough for MALP (one row per check); a
// frame whose cut list grows past it (ALP, or MALP continued as ALP) moves
// to a wide workspace in global scratch. Row indices are packed in 15 bits
// and column indices n + r in 16.
int rows_cap(const lpdec_params& prm, int n, int m) {
    long long cap = prm.lp_rows_cap > 0 ? prm.lp_rows_cap : 2LL * m;
    cap = std::min<long long>({cap, 32767LL, 65535LL - n});
    return (int)std::max<long long>(cap, 1);
}

CodeView view_of(const lpdec_code* c, const lpdec_params& prm) {
    CodeView v;
    v.n = c->n; v.m = c->m; v.E = c->E;
    v.pwide = rows_cap(prm, c->n, c->m);
    v.pmax = std::min(v.pwide, c->m);   // MALP: one row per check
    v.eamax = v.pmax * c->dmax;
    v.eawide = v.pwide * c->dmax;
    v.h_ptr = c->h_ptr; v.h_col = c->h_col; v.e_chk = c->e_chk;
    v.v_ptr = c->v_ptr; v.v_chk = c->v_chk; v.v_eidx = c->v_eidx;
    return v;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Every array of the layout lies inside its region (shared or global), is
// 16-byte aligned and overlaps no other array.
bool layout_ok(const Layout& L, const std::vector<size_t>& sizes) {
    struct Iv { size_t a, b; bool g; };
    std::vector<Iv> iv;
    for (int k = 0; k < A_COUNT; ++k) {
        bool g = (L.off[k] & kGlobalBit) != 0;
        size_t a = L.off[k] & ~kGlobalBit;
        if (a % 16) return false;
        iv.push_back({a, a + sizes[k], g});
        if (!g && a + sizes[k] > L.smem_bytes) return false;
        if (g && a + sizes[k] > L.gbytes) return false;
    }
    for (size_t i = 0; i < iv.size(); ++i)
        for (size_t j = i + 1; j < iv.size(); ++j)
            if (iv[i].g == iv[j].g && iv[i].a < iv[j].b && iv[j].a < iv[i].b &&
                iv[i].b > iv[i].a && iv[j].b > iv[j].a)
                return false;
    return true;
}

// Capacities one workspace is laid out for: the largest code of a launch.
struct Dims {
    int n = 0, m = 0, pmax = 0, eamax = 0, pwide = 0, eawide = 0;
    void cover(const CodeView& v) {
        n = std::max(n, v.n); m = std::max(m, v.m);
        pmax = std::max(pmax, v.pmax); eamax = std::max(eamax, v.eamax);
        pwide = std::max(pwide, v.pwide); eawide = std::max(eawide, v.eawide);
    }
};

// Largest LP (rows) for which the dense Cholesky fallback keeps its FP64
// matrix in per-CTA scratch (32 MB at the limit).
constexpr int kDenseMaxRows = 2048;

// Lays the workspace out. Hot arrays (everything the PCG loop and the MTS
// selection touch) go to shared memory in priority order while they fit the
// budget; the bitmap and the level pointer arrays, which the kernels update
// with shared-memory atomics, always do. The FP64 interior-point state goes
// to per-CTA global scratch. dense_rows = capacity of the dense fallback's
// matrix (0 = fallback off).
Layout make_layout(const Dims& d, size_t budget, size_t real_bytes, bool m32, int dense_rows,
                   bool all_global = false) {
    const int n = d.n, m = d.m, pm = d.pmax;
    const size_t ea = (size_t)std::max(d.eamax, 1);
    const size_t q = (size_t)n + pm;
    size_t q2 = 1;
    while (q2 < q) q2 <<= 1;
    const size_t vec = vec_hot_bytes(n, pm, real_bytes, m32);
    const size_t vecc = vec_cold_bytes(n, pm, real_bytes, q2);
    struct Spec { int id; size_t bytes; int where; };  // 0 = budgeted, 1 = always shared, 2 = global
    const size_t D = 8, I = 4, H = 2, P = (size_t)pm;
    std::vector<Spec> specs = {
        {S_BITMAP, I * ((q + 31) / 32), 1}, {S_LBPTR, I * (P + 2), 1}, {S_LFPTR, I * (P + 2), 1},
        {S_CUR, I * (P + 2), 1},
        // budgeted arrays in priority order: first what every PCG iteration
        // reads on its serial path (the two level-scheduled triangular
        // solves: right side, solution and pivot scaling, dependency lists
        // and ranges, level rows, pivot signs), then what the serial greedy
        // of the MTS selection walks once per interior-point iteration
        // (pivots, degrees, levels, the column and row entries of A), then
        // the rest of the level build, then the cut search and the cut
        // list, and last the vectors only the parallel passes touch (and
        // the sort keys)
        {S_VEC, vec, 0}, {S_BDEP, H * ea, 0}, {S_FDEP, H * ea, 0}, {S_LBSE, 8 * P, 0},
        {S_LFSE, 8 * P, 0}, {S_LBROWS, H * P, 0}, {S_LFROWS, H * P, 0}, {S_PSGN, P, 0},
        {S_PIVCOL, H * P, 0}, {S_PIVROW, H * q, 0}, {S_LF, H * P, 0}, {S_LB, H * P, 0},
        {S_DEG, H * q, 0}, {S_SELROW, H * P, 0},
        {S_CPTR, I * ((size_t)n + 1), 0}, {S_ROWENT, H * ea, 0}, {S_RPTR, I * (P + 1), 0},
        {S_COLENT, H * ea, 0},
        {S_BPTR, I * (P + 1), 0}, {S_FPTR, I * (P + 1), 0},
        {S_HPTR, I * ((size_t)m + 1), 0}, {S_VPTR, I * ((size_t)n + 1), 0},
        {S_CCHK, H * P, 0}, {S_CRPTR, I * ((size_t)m + 1), 0}, {S_FLAGS, (size_t)m, 0},
        {S_MASK, I * (size_t)m, 0}, {S_CMASK, I * P, 0}, {S_CACT, P, 0},
        {S_FLIP, I * (((size_t)n + 31) / 32), 0}, {S_VECC, vecc, 0},
        {G_X, D * q, 2}, {G_Z, D * q, 2}, {G_RC, D * q, 2}, {G_D2, D * q, 2}, {G_Y, D * P, 2},
        {G_B, D * P, 2}, {G_W, D * P, 2}, {G_DY, D * P, 2}, {G_R64, D * P, 2}, {G_U, D * n, 2},
        {G_T64, D * n, 2}, {G_BASIC, q, 2},
        {G_VX, D * q, 2}, {G_V1, D * q, 2}, {G_V2, D * q, 2}, {G_V3, D * q, 2}, {G_V4, D * q, 2},
        {G_VR1, D * P, 2}, {G_VR2, D * P, 2},
        {G_P64, real_bytes < 8 ? D * vec_elems(n, pm) : 16, 2},
        {G_QD, dense_rows > 0 ? D * (size_t)dense_rows * dense_rows : 16, 2},
        {G_CCHK2, H * P, 2}, {G_CMASK2, I * P, 2}, {G_CRPTR2, I * ((size_t)m + 1), 2},
        {G_GAM, D * (size_t)n, 2}, {G_LZ, D * (2 * (size_t)kLz + 2), 2},
        {G_XW, D * q, 2}, {G_ZW, D * q, 2}, {G_YW, D * P, 2}, {G_PROW, I * (size_t)m, 2},
        {G_PMASK, I * (size_t)m, 2},
    };
    Layout L{};
    size_t s = 0, g = 0;
    std::vector<size_t> sizes(A_COUNT, 0);
    for (const auto& sp : specs) {
        size_t b = align_up(sp.bytes, 16);
        sizes[sp.id] = sp.bytes;
        if (!all_global && (sp.where == 1 || (sp.where == 0 && s + b <= budget))) {
            L.off[sp.id] = (uint32_t)s;
            s += b;
        } else {
            L.off[sp.id] = (uint32_t)g | kGlobalBit;
            g += b;
        }
    }
    L.smem_bytes = (uint32_t)s;
    L.q2 = (uint32_t)q2;
    L.dense = (uint32_t)std::max(dense_rows, 0);
    L.nmax = (uint32_t)n;
    L.mmax = (uint32_t)m;
    L.pmax = (uint32_t)pm;
    L.gbytes = align_up(g, 256);
    L.stride = L.gbytes;
    if (specs.size() != (size_t)A_COUNT || !layout_ok(L, sizes) || g >= kGlobalBit)
        L.smem_bytes = 0xffffffffu;
    return L;
}

// Rows of the dense fallback's matrix: the main capacity and a quarter more
// (frames continued as ALP); off for codes whose main capacity exceeds 2048
// rows (its matrix would not be worth its memory).
int dense_rows_for(const Dims& d) {
    if (d.pmax > kDenseMaxRows) return 0;
    return std::min({d.pmax + d.pmax / 4, std::max(d.pwide, d.pmax), kDenseMaxRows});
}

// The wide workspace (all in global scratch) for frames whose cut list
// outgrows the main one; gbytes = 0 when the capacity does not exceed it.
Layout make_wide_layout(const Dims& d, size_t real_bytes, bool m32) {
    Layout W{};
    if (d.pwide <= d.pmax) return W;
    Dims w = d;
    w.pmax = d.pwide;
    w.eamax = d.eawide;
    W = make_layout(w, 0, real_bytes, m32, 0, true);
    return W;
}

// Both workspaces of a launch: main (L) then wide (Lw) in each CTA's scratch.
bool make_layouts(const Dims& d, size_t budget, size_t real_bytes, bool m32, int dense_rows,
                  Layout* L, Layout* Lw) {
    *L = make_layout(d, budget, real_bytes, m32, dense_rows);
    *Lw = make_wide_layout(d, real_bytes, m32);
    if (L->smem_bytes == 0xffffffffu || Lw->smem_bytes == 0xffffffffu) return false;
    L->stride = L->gbytes + Lw->gbytes;
    Lw->stride = L->stride;
    return true;
}

struct Launch {
    Layout L, Lw;
    int threads;
    int grid;
};

size_t smem_budget_of(const lpdec_ctx* ctx) {
    size_t cap = (size_t)ctx->smem_optin - sizeof(KernelShared) - 1024;
    // Library choice: a third of the SM's shared memory per CTA, so that three
    // frames share an SM (the frame's chain of dependent block-wide steps
    // leaves the SM mostly idle; measured 27% more frames/s than two CTAs of
    // the maximal layout on the n=1008 workload). Arrays that do not fit go
    // to global scratch, in the layout's priority order.
    const size_t third = (size_t)ctx->smem_per_sm / 3;
    const size_t per_cta = sizeof(KernelShared) + 1024 + 256;
    return ctx->prm.smem_budget > 0 ? std::min((size_t)ctx->prm.smem_budget, cap)
         : (third > per_cta ? std::min(cap, third - per_cta) : cap);
}

// Layout, CTA size and grid of a launch (no allocation); *per_sm = CTAs per SM.
template <typename K>
int32_t shape(lpdec_ctx* ctx, const Dims& dims, int nframes, K kernel, size_t real_bytes,
              Launch* out, int* per_sm_out) {
    int threads = ctx->prm.threads_per_block > 0 ? ctx->prm.threads_per_block : 128;
    threads = std::max(32, std::min(512, threads / 32 * 32));
    Layout L, Lw;
    if (!make_layouts(dims, smem_budget_of(ctx), real_bytes, ctx->prm.precision == LPDEC_M32,
                      dense_rows_for(dims), &L, &Lw)) {
        snprintf(g_err, sizeof g_err, "inconsistent workspace layout");
        return LPDEC_ERR_INVALID_ARG;
    }
    if (L.smem_bytes + sizeof(KernelShared) > (size_t)ctx->smem_optin) {
        snprintf(g_err, sizeof g_err, "frame needs %u bytes of shared memory", L.smem_bytes);
        return LPDEC_ERR_INVALID_ARG;
    }
    CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, L.smem_bytes));
    if (per_sm < 1) {
        snprintf(g_err, sizeof g_err, "kernel does not fit on an SM");
        return LPDEC_ERR_INVALID_ARG;
    }
    out->L = L;
    out->Lw = Lw;
    out->threads = threads;
    out->grid = std::max(1, std::min(nframes, per_sm * ctx->sm_count));
    *per_sm_out = per_sm;
    return LPDEC_OK;
}

template <typename K>
int32_t plan(lpdec_ctx* ctx, const Dims& dims, int nframes, K kernel, size_t real_bytes,
             Launch* out) {
    int per_sm = 0;
    int32_t rc = shape(ctx, dims, nframes, kernel, real_bytes, out, &per_sm);
    if (rc != LPDEC_OK) return rc;
    const Layout& L = out->L;
    const int grid = out->grid;
    // scratch for the full grid, whatever this batch needs, so that a small
    // batch (a warm-up) leaves no allocation to a later, larger one
    size_t need = (size_t)per_sm * ctx->sm_count * L.stride;
    if (ctx->budget && need + ctx->staging_bytes > ctx->budget) need = (size_t)grid * L.stride;
    if (need > ctx->gscratch_bytes) {
        if (ctx->budget && need + ctx->staging_bytes > ctx->budget) return LPDEC_ERR_OUT_OF_BUDGET;
        if (ctx->gscratch) CK(cudaFree(ctx->gscratch));
        ctx->gscratch = nullptr;
        ctx->gscratch_bytes = 0;
        CK(cudaMalloc(&ctx->gscratch, need));
        ctx->gscratch_bytes = need;
    }
    return LPDEC_OK;
}

template <typename K>
int32_t plan(lpdec_ctx* ctx, const lpdec_code* code, int nframes, K kernel, size_t real_bytes,
             Launch* out) {
    Dims d;
    d.cover(view_of(code, ctx->prm));
    return plan(ctx, d, nframes, kernel, real_bytes, out);
}

int32_t staging(lpdec_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->staging_bytes) return LPDEC_OK;
    if (ctx->budget && bytes + ctx->gscratch_bytes > ctx->budget) return LPDEC_ERR_OUT_OF_BUDGET;
    if (ctx->staging) CK(cudaFree(ctx->staging));
    ctx->staging = nullptr;
    ctx->staging_bytes = 0;
    CK(cudaMalloc(&ctx->staging, bytes));
    ctx->staging_bytes = bytes;
    return LPDEC_OK;
}

// Device and pinned host buffers for the metadata of a mixed batch (grown,
// never shrunk; the host copy is reused only after its last copy ran).
int32_t meta_buffers(lpdec_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->meta_bytes) return LPDEC_OK;
    if (ctx->meta_done) CK(cudaEventSynchronize(ctx->meta_done));
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_meta);
    cudaFreeHost(ctx->h_meta);
    ctx->d_meta = ctx->h_meta = nullptr;
    ctx->meta_bytes = 0;
    bytes = align_up(bytes * 2, 4096);
    CK(cudaMalloc(&ctx->d_meta, bytes));
    CK(cudaMallocHost(&ctx->h_meta, bytes));
    ctx->meta_bytes = bytes;
    return LPDEC_OK;
}

int32_t host_staging(lpdec_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->h_stage_bytes) return LPDEC_OK;
    cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    CK(cudaMallocHost(&ctx->h_stage, bytes));
    ctx->h_stage_bytes = bytes;
    return LPDEC_OK;
}

// Whether a one-code batch of nframes on `grid` CTAs is handed out in the
// hardest-first order (lpdec_params.order_frames).
bool orders_frames(const lpdec_params& p, int nframes, int grid) {
    return (p.order_frames == 2 || (p.order_frames == 1 && nframes > grid)) &&
           nframes <= (int)kOrderIdx;
}

bool params_ok(const lpdec_params& p) {
    if (p.variant != LPDEC_MALP_A && p.variant != LPDEC_MALP_B && p.variant != LPDEC_ALP)
        return false;
    if (p.precision != LPDEC_FP64 && p.precision != LPDEC_MIXED && p.precision != LPDEC_M32)
        return false;
    if (p.precond < LPDEC_MTS_COLUMN || p.precond > LPDEC_MTS_ROWWISE_TRI) return false;
    if (p.lane_policy != 0 && p.lane_policy != 1 && p.lane_policy != 2 && p.lane_policy != 4 &&
        p.lane_policy != 8)
        return false;
    if (p.order_frames < 0 || p.order_frames > 2) return false;
    if (p.dense_switch < 0) return false;
    return p.lp_rows_cap >= 0;
}

int32_t check_ctx_code(lpdec_ctx* ctx, const lpdec_code* code) {
    if (!ctx || !code || code->device != ctx->device) {
        snprintf(g_err, sizeof g_err, "null context/code, or a code of another device");
        return LPDEC_ERR_INVALID_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    return LPDEC_OK;
}

int32_t launch_decode(lpdec_ctx* ctx, const lpdec_code* code, int nframes, const double* d_gamma,
                      double* d_u, uint8_t* d_hard, int32_t* d_cert, uint32_t* d_mask,
                      lpdec_stats* d_stats, cudaStream_t s) {
    if (nframes == 0) return LPDEC_OK;
    Launch ln;
    const bool mixed = ctx->prm.precision == LPDEC_MIXED;
    int32_t rc = mixed ? plan(ctx, code, nframes, k_decode<float>, 4, &ln)
                       : plan(ctx, code, nframes, k_decode<double>, 8, &ln);
    if (rc) return rc;
    const CodeView cv = view_of(code, ctx->prm);
    const DevParams dp = to_dev(ctx->prm);
    // hardest-first frame order when frames queue behind the grid
    const unsigned long long* order = nullptr;
    if (orders_frames(ctx->prm, nframes, ln.grid)) {
        int n2 = 1;
        while (n2 < nframes) n2 <<= 1;
        if ((size_t)n2 > ctx->order_n) {
            if (ctx->d_order) CK(cudaFree(ctx->d_order));
            ctx->d_order = nullptr;
            ctx->order_n = 0;
            CK(cudaMalloc(&ctx->d_order, (size_t)n2 * sizeof(unsigned long long)));
            ctx->order_n = (size_t)n2;
        }
        k_order_keys<<<std::min(1024, (n2 + 7) / 8), 256, 0, s>>>(d_gamma, code->n, nframes, n2,
                                                                 ctx->d_order);
        k_sort_keys<<<1, 1024, 0, s>>>(ctx->d_order, n2);
        CK(cudaGetLastError());
        order = ctx->d_order;
    }
    CK(cudaMemsetAsync(ctx->counter, 0, sizeof(int), s));
    if (mixed)
        k_decode<float><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
            cv, nullptr, nullptr, dp, ln.L, ln.Lw, d_gamma, d_u, d_hard, d_cert, d_mask, d_stats,
            nframes, ctx->counter, ctx->gscratch, order);
    else
        k_decode<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
            cv, nullptr, nullptr, dp, ln.L, ln.Lw, d_gamma, d_u, d_hard, d_cert, d_mask, d_stats,
            nframes, ctx->counter, ctx->gscratch, order);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

// Batch of frames of several codes (ragged frame-major arrays, descriptors
// built here). The code table and the descriptors go to the context's
// device buffer through its pinned host buffer, on stream s.
int32_t launch_decode_mixed(lpdec_ctx* ctx, int nframes, const lpdec_code* const* codes,
                            const double* d_gamma, double* d_u, uint8_t* d_hard, int32_t* d_cert,
                            uint32_t* d_mask, lpdec_stats* d_stats, cudaStream_t s) {
    if (nframes == 0) return LPDEC_OK;
    std::vector<const lpdec_code*> table;
    std::vector<FrameDesc> desc((size_t)nframes);
    Dims dims;
    long long on = 0, om = 0;
    for (int f = 0; f < nframes; ++f) {
        const lpdec_code* c = codes[f];
        int k = -1;
        for (size_t t = 0; t < table.size(); ++t)
            if (table[t] == c) { k = (int)t; break; }
        if (k < 0) {
            k = (int)table.size();
            table.push_back(c);
            dims.cover(view_of(c, ctx->prm));
        }
        desc[f] = FrameDesc{k, 0, on, om};
        on += c->n;
        om += c->m;
    }
    std::vector<CodeView> views;
    for (const lpdec_code* c : table) views.push_back(view_of(c, ctx->prm));
    const size_t vbytes = align_up(views.size() * sizeof(CodeView), 256);
    const size_t dbytes = desc.size() * sizeof(FrameDesc);
    int32_t rc = meta_buffers(ctx, vbytes + dbytes);
    if (rc) return rc;
    // the pinned buffer may still feed the previous launch's copy
    CK(cudaEventSynchronize(ctx->meta_done));
    std::memcpy(ctx->h_meta, views.data(), views.size() * sizeof(CodeView));
    std::memcpy(ctx->h_meta + vbytes, desc.data(), dbytes);
    CK(cudaMemcpyAsync(ctx->d_meta, ctx->h_meta, vbytes + dbytes, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(ctx->meta_done, s));
    Launch ln;
    const bool mixed = ctx->prm.precision == LPDEC_MIXED;
    rc = mixed ? plan(ctx, dims, nframes, k_decode<float>, 4, &ln)
               : plan(ctx, dims, nframes, k_decode<double>, 8, &ln);
    if (rc) return rc;
    const CodeView* dv = reinterpret_cast<const CodeView*>(ctx->d_meta);
    const FrameDesc* dd = reinterpret_cast<const FrameDesc*>(ctx->d_meta + vbytes);
    const DevParams dp = to_dev(ctx->prm);
    CK(cudaMemsetAsync(ctx->counter, 0, sizeof(int), s));
    if (mixed)
        k_decode<float><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
            views[0], dv, dd, dp, ln.L, ln.Lw, d_gamma, d_u, d_hard, d_cert, d_mask, d_stats,
            nframes,
            ctx->counter, ctx->gscratch, nullptr);
    else
        k_decode<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
            views[0], dv, dd, dp, ln.L, ln.Lw, d_gamma, d_u, d_hard, d_cert, d_mask, d_stats,
            nframes,
            ctx->counter, ctx->gscratch, nullptr);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

}  // namespace

extern "C" {

void lpdec_default_params(lpdec_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->sigma = 0.1;
    p->eta = 0.99;
    p->tol_gap = 1e-8;
    p->tol_feas = 1e-8;
    p->tol_pcg = 1e-10;
    p->tau_act = 1e-9;
    p->tau_cut = 1e-9;
    p->tau_int = 1e-9;
    p->pcg_gap_factor = 0.01;
    p->tol_inner = 1e-5;
    p->tol_feas_loose = 1e-6;
    p->tol_cert = 1e-3;
    p->tau_inc = 1e-9;
    p->max_alp = 200;
    p->max_ipm = 60;
    p->max_pcg = 1000;
    p->variant = LPDEC_MALP_A;
    p->precision = LPDEC_FP64;
    p->lp_rows_cap = 0;
    p->precond = LPDEC_MTS_COLUMN;
    p->precond_switch = 150;
    p->warm_start = 0;
    p->mts_reuse = 0;
    p->lane_policy = 0;
    p->order_frames = 1;
    p->dense_switch = 64;
    p->reserved = 0;
}

const char* lpdec_error_string(int32_t code) {
    switch (code) {
        case LPDEC_OK: return "ok";
        case LPDEC_ERR_INVALID_ARG: return "invalid argument";
        case LPDEC_ERR_OUT_OF_BUDGET: return "out of HBM budget or LP row capacity";
        case LPDEC_ERR_NOT_CONVERGED: return "iteration cap reached";
        case LPDEC_ERR_TIMEOUT: return "timeout";
        case LPDEC_ERR_PENDING: return "pending";
        case LPDEC_ERR_CUDA: return g_err[0] ? g_err : "CUDA error";
        case LPDEC_ERR_NO_DEVICE: return "no usable CUDA device";
        case LPDEC_ERR_CANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

int32_t lpdec_workspace_bytes(int32_t m, int32_t n, int32_t E, int32_t precision,
                              int32_t smem_budget, size_t* smem_bytes,
                              size_t* global_bytes_per_frame) {
    if (m <= 0 || n <= 0 || m > 32767 || n > 32767 || E <= 0 || E > 32 * m ||
        (precision != LPDEC_FP64 && precision != LPDEC_MIXED && precision != LPDEC_M32))
        return LPDEC_ERR_INVALID_ARG;
    size_t budget = smem_budget > 0 ? (size_t)smem_budget : (size_t)227 * 1024;
    lpdec_params prm;
    lpdec_default_params(&prm);
    Dims d;
    d.n = n;
    d.m = m;
    const int dmax = (E + m - 1) / m;   // check degrees at most ceil(E/m)
    d.pwide = rows_cap(prm, n, m);
    d.pmax = std::min(d.pwide, m);
    d.eamax = d.pmax * dmax;
    d.eawide = d.pwide * dmax;
    Layout L, Lw;
    if (!make_layouts(d, budget, precision == LPDEC_MIXED ? 4 : 8, precision == LPDEC_M32,
                      dense_rows_for(d), &L, &Lw))
        return LPDEC_ERR_INVALID_ARG;
    if (L.smem_bytes == 0xffffffffu) return LPDEC_ERR_INVALID_ARG;
    if (smem_bytes) *smem_bytes = L.smem_bytes + sizeof(KernelShared);
    if (global_bytes_per_frame) *global_bytes_per_frame = (size_t)L.stride;
    return LPDEC_OK;
}

int32_t lpdec_batch_grid(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                         int32_t* grid, int32_t* ordered) {
    if (!ctx || !code || !grid || nframes < 0 || code->device != ctx->device)
        return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->device));
    Dims d;
    d.cover(view_of(code, ctx->prm));
    Launch ln;
    int per_sm = 0;
    const bool mixed = ctx->prm.precision == LPDEC_MIXED;
    int32_t rc = mixed ? shape(ctx, d, nframes, k_decode<float>, 4, &ln, &per_sm)
                       : shape(ctx, d, nframes, k_decode<double>, 8, &ln, &per_sm);
    if (rc != LPDEC_OK) return rc;
    *grid = nframes > 0 ? ln.grid : 0;
    if (ordered) *ordered = nframes > 0 && orders_frames(ctx->prm, nframes, ln.grid);
    return LPDEC_OK;
}

int32_t lpdec_ctx_create(int32_t device, const lpdec_params* params, size_t hbm_budget_bytes,
                         lpdec_ctx** out) {
    if (!out) return LPDEC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= device || device < 0) {
        cudaGetLastError();
        snprintf(g_err, sizeof g_err, "no CUDA device %d", device);
        return LPDEC_ERR_NO_DEVICE;
    }
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) {
        snprintf(g_err, sizeof g_err, "device %d is sm_%d%d; the library is compiled for sm_103a",
                 device, prop.major, prop.minor);
        return LPDEC_ERR_NO_DEVICE;
    }
    CK(cudaSetDevice(device));
    lpdec_ctx* c = new (std::nothrow) lpdec_ctx();
    if (!c) return LPDEC_ERR_INVALID_ARG;
    c->device = device;
    if (params) c->prm = *params; else lpdec_default_params(&c->prm);
    if (!params_ok(c->prm)) {
        delete c;
        return LPDEC_ERR_INVALID_ARG;
    }
    c->budget = hbm_budget_bytes;
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = (int)prop.sharedMemPerBlockOptin;
    c->smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->meta_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&c->counter, sizeof(int)) != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "context allocation failed");
        if (c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return LPDEC_ERR_CUDA;
    }
    *out = c;
    return LPDEC_OK;
}

void lpdec_ctx_destroy(lpdec_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->meta_done) cudaEventSynchronize(ctx->meta_done);
    cudaFree(ctx->gscratch);
    cudaFree(ctx->staging);
    cudaFree(ctx->counter);
    cudaFree(ctx->d_meta);
    cudaFree(ctx->d_order);
    cudaFreeHost(ctx->h_meta);
    cudaFreeHost(ctx->h_stage);
    if (ctx->meta_done) cudaEventDestroy(ctx->meta_done);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int32_t lpdec_ctx_set_params(lpdec_ctx* ctx, const lpdec_params* params) {
    if (!ctx || !params) return LPDEC_ERR_INVALID_ARG;
    if (!params_ok(*params)) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->prm = *params;
    return LPDEC_OK;
}

int32_t lpdec_code_create(lpdec_ctx* ctx, int32_t m, int32_t n, const int32_t* row_ptr,
                          const int32_t* col_idx, lpdec_code** out) {
    if (!ctx || !out || !row_ptr || m <= 0 || n <= 0 || m > 32767 || n > 32767)
        return LPDEC_ERR_INVALID_ARG;
    *out = nullptr;
    if (row_ptr[0] != 0) return LPDEC_ERR_INVALID_ARG;
    for (int j = 0; j < m; ++j) {
        int d = row_ptr[j + 1] - row_ptr[j];
        if (d < 1 || d > 32) return LPDEC_ERR_INVALID_ARG;
    }
    const int E = row_ptr[m];
    if (E > 0 && !col_idx) return LPDEC_ERR_INVALID_ARG;
    int dmax = 0;
    for (int j = 0; j < m; ++j) dmax = std::max(dmax, row_ptr[j + 1] - row_ptr[j]);
    std::vector<int> e_chk(E), vdeg(n + 1, 0);
    for (int j = 0; j < m; ++j) {
        for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
            int i = col_idx[e];
            if (i < 0 || i >= n) return LPDEC_ERR_INVALID_ARG;
            if (e > row_ptr[j] && col_idx[e - 1] >= i) return LPDEC_ERR_INVALID_ARG;
            e_chk[e] = j;
            vdeg[i + 1]++;
        }
    }
    std::vector<int> v_ptr(n + 1, 0), v_chk(E), v_eidx(E);
    for (int i = 0; i < n; ++i) v_ptr[i + 1] = v_ptr[i] + vdeg[i + 1];
    std::vector<int> fill(v_ptr.begin(), v_ptr.end() - 1);
    for (int j = 0; j < m; ++j)
        for (int e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
            int i = col_idx[e];
            v_chk[fill[i]] = j;
            v_eidx[fill[i]] = e;
            fill[i]++;
        }
    CK(cudaSetDevice(ctx->device));
    lpdec_code* c = new (std::nothrow) lpdec_code();
    if (!c) return LPDEC_ERR_INVALID_ARG;
    c->ctx = ctx;
    c->device = ctx->device;
    c->m = m; c->n = n; c->E = E;
    c->dmax = dmax;
    auto up = [&](int** dst, const int* src, size_t cnt) -> bool {
        if (cudaMalloc(dst, std::max<size_t>(cnt, 1) * sizeof(int)) != cudaSuccess) return false;
        return cnt == 0 || cudaMemcpy(*dst, src, cnt * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = up(&c->h_ptr, row_ptr, m + 1) && up(&c->h_col, col_idx, E) &&
              up(&c->e_chk, e_chk.data(), E) && up(&c->v_ptr, v_ptr.data(), n + 1) &&
              up(&c->v_chk, v_chk.data(), E) && up(&c->v_eidx, v_eidx.data(), E);
    if (!ok) {
        snprintf(g_err, sizeof g_err, "code upload failed");
        lpdec_code_destroy(c);
        return LPDEC_ERR_CUDA;
    }
    *out = c;
    return LPDEC_OK;
}

void lpdec_code_destroy(lpdec_code* code) {
    if (!code) return;
    if (code->ctx) cudaSetDevice(code->ctx->device);
    cudaFree(code->h_ptr); cudaFree(code->h_col); cudaFree(code->e_chk);
    cudaFree(code->v_ptr); cudaFree(code->v_chk); cudaFree(code->v_eidx);
    delete code;
}

int32_t lpdec_decode_batch_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                                  const double* d_gamma, double* d_u, uint8_t* d_hard,
                                  int32_t* d_cert, uint32_t* d_cut_mask, lpdec_stats* d_stats,
                                  void* stream) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 0 || (nframes > 0 && (!d_gamma || !d_u || !d_hard || !d_cert)))
        return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    return launch_decode(ctx, code, nframes, d_gamma, d_u, d_hard, d_cert, d_cut_mask, d_stats,
                         (cudaStream_t)stream);
}

int32_t lpdec_decode_frames(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                            const double* gamma, double* u_out, uint8_t* hard_out,
                            int32_t* cert_out, uint32_t* cut_mask_out, lpdec_stats* stats) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 0 || (nframes > 0 && (!gamma || !u_out || !hard_out || !cert_out)))
        return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    for (size_t k = 0; k < (size_t)nframes * code->n; ++k)
        if (!std::isfinite(gamma[k])) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    const size_t nf = (size_t)nframes, n = code->n, m = code->m;
    size_t o_g = 0;
    size_t o_u = align_up(o_g + nf * n * 8, 256);
    size_t o_h = align_up(o_u + nf * n * 8, 256);
    size_t o_c = align_up(o_h + nf * n, 256);
    size_t o_m = align_up(o_c + nf * 4, 256);
    size_t o_s = align_up(o_m + nf * m * 4, 256);
    size_t tot = align_up(o_s + nf * sizeof(lpdec_stats), 256);
    rc = staging(ctx, tot);
    if (rc) return rc;
    char* b = ctx->staging;
    cudaStream_t s = ctx->stream;
    CK(cudaMemcpyAsync(b + o_g, gamma, nf * n * 8, cudaMemcpyHostToDevice, s));
    rc = launch_decode(ctx, code, nframes, (const double*)(b + o_g), (double*)(b + o_u),
                       (uint8_t*)(b + o_h), (int32_t*)(b + o_c),
                       cut_mask_out ? (uint32_t*)(b + o_m) : nullptr,
                       stats ? (lpdec_stats*)(b + o_s) : nullptr, s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(u_out, b + o_u, nf * n * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hard_out, b + o_h, nf * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(cert_out, b + o_c, nf * 4, cudaMemcpyDeviceToHost, s));
    if (cut_mask_out) CK(cudaMemcpyAsync(cut_mask_out, b + o_m, nf * m * 4, cudaMemcpyDeviceToHost, s));
    if (stats) CK(cudaMemcpyAsync(stats, b + o_s, nf * sizeof(lpdec_stats), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return LPDEC_OK;
}

int32_t lpdec_decode(lpdec_ctx* ctx, const lpdec_code* code, const double* gamma, double* u_out,
                     uint8_t* hard_out, int32_t* cert_out, uint32_t* cut_mask_out,
                     lpdec_stats* stats) {
    return lpdec_decode_frames(ctx, code, 1, gamma, u_out, hard_out, cert_out, cut_mask_out, stats);
}

// Frames of several codes: checks, packs the per-frame host arrays into the
// context's pinned buffer, runs one persistent launch over the ragged batch
// and scatters the results back.
int32_t lpdec_decode_batch(lpdec_ctx* ctx, int32_t nframes, const lpdec_code* const* codes,
                           const double* const* gammas, double* const* u_out,
                           uint8_t* const* hard_out, int32_t* cert_out,
                           uint32_t* const* cut_mask_out, lpdec_stats* stats) {
    if (!ctx || nframes < 0) return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    if (!codes || !gammas || !u_out || !hard_out || !cert_out) return LPDEC_ERR_INVALID_ARG;
    size_t N = 0, M = 0;
    for (int f = 0; f < nframes; ++f) {
        int32_t rc = check_ctx_code(ctx, codes[f]);
        if (rc) return rc;
        if (!gammas[f] || !u_out[f] || !hard_out[f]) return LPDEC_ERR_INVALID_ARG;
        for (int i = 0; i < codes[f]->n; ++i)
            if (!std::isfinite(gammas[f][i])) return LPDEC_ERR_INVALID_ARG;
        N += codes[f]->n;
        M += codes[f]->m;
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    const size_t nf = (size_t)nframes;
    size_t o_g = 0;
    size_t o_u = align_up(o_g + N * 8, 256);
    size_t o_h = align_up(o_u + N * 8, 256);
    size_t o_c = align_up(o_h + N, 256);
    size_t o_m = align_up(o_c + nf * 4, 256);
    size_t o_s = align_up(o_m + M * 4, 256);
    size_t tot = align_up(o_s + nf * sizeof(lpdec_stats), 256);
    int32_t rc = staging(ctx, tot);
    if (rc) return rc;
    rc = host_staging(ctx, tot);
    if (rc) return rc;
    char* b = ctx->staging;
    char* h = ctx->h_stage;
    cudaStream_t s = ctx->stream;
    for (size_t f = 0, on = 0; f < nf; on += codes[f]->n, ++f)
        std::memcpy(h + o_g + on * 8, gammas[f], (size_t)codes[f]->n * 8);
    CK(cudaMemcpyAsync(b + o_g, h + o_g, N * 8, cudaMemcpyHostToDevice, s));
    rc = launch_decode_mixed(ctx, nframes, codes, (const double*)(b + o_g), (double*)(b + o_u),
                             (uint8_t*)(b + o_h), (int32_t*)(b + o_c), (uint32_t*)(b + o_m),
                             (lpdec_stats*)(b + o_s), s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h + o_u, b + o_u, tot - o_u, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (size_t f = 0, on = 0, om = 0; f < nf; on += codes[f]->n, om += codes[f]->m, ++f) {
        const size_t n = codes[f]->n, m = codes[f]->m;
        std::memcpy(u_out[f], h + o_u + on * 8, n * 8);
        std::memcpy(hard_out[f], h + o_h + on, n);
        if (cut_mask_out && cut_mask_out[f]) std::memcpy(cut_mask_out[f], h + o_m + om * 4, m * 4);
    }
    std::memcpy(cert_out, h + o_c, nf * 4);
    if (stats) std::memcpy(stats, h + o_s, nf * sizeof(lpdec_stats));
    return LPDEC_OK;
}

int32_t lpdec_decode_mixed_device(lpdec_ctx* ctx, int32_t nframes, const lpdec_code* const* codes,
                                  const double* d_gamma, double* d_u, uint8_t* d_hard,
                                  int32_t* d_cert, uint32_t* d_cut_mask, lpdec_stats* d_stats,
                                  void* stream) {
    if (!ctx || nframes < 0) return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    if (!codes || !d_gamma || !d_u || !d_hard || !d_cert) return LPDEC_ERR_INVALID_ARG;
    for (int f = 0; f < nframes; ++f) {
        int32_t rc = check_ctx_code(ctx, codes[f]);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    return launch_decode_mixed(ctx, nframes, codes, d_gamma, d_u, d_hard, d_cert, d_cut_mask,
                               d_stats, (cudaStream_t)stream);
}

// Picks the warp-mode sweep schedule (lanes per row) for this context and
// code: decodes the sample once per candidate and keeps the one with the
// least total device time of the frames on their CTAs (the sum of
// stats.seconds, which a launch's slowest frame does not dominate).
int32_t lpdec_autotune(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                       const double* gamma, int32_t* policy_out, double* seconds_out) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 1 || !gamma) return LPDEC_ERR_INVALID_ARG;
    for (size_t k = 0; k < (size_t)nframes * code->n; ++k)
        if (!std::isfinite(gamma[k])) return LPDEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    const size_t nf = (size_t)nframes, n = code->n;
    const size_t o_g = 0, o_u = align_up(nf * n * 8, 256), o_h = align_up(o_u + nf * n * 8, 256);
    const size_t o_c = align_up(o_h + nf * n, 256), o_s = align_up(o_c + nf * 4, 256);
    const size_t tot = align_up(o_s + nf * sizeof(lpdec_stats), 256);
    rc = staging(ctx, tot);
    if (rc) return rc;
    char* b = ctx->staging;
    cudaStream_t s = ctx->stream;
    CK(cudaMemcpyAsync(b + o_g, gamma, nf * n * 8, cudaMemcpyHostToDevice, s));
    std::vector<lpdec_stats> st(nf);
    const int cand[5] = {0, 1, 2, 4, 8};
    const int keep = ctx->prm.lane_policy;
    int best = keep;
    double best_t = INFINITY;
    for (int k = 0; k < 5; ++k) {
        ctx->prm.lane_policy = cand[k];
        rc = launch_decode(ctx, code, nframes, (const double*)(b + o_g), (double*)(b + o_u),
                           (uint8_t*)(b + o_h), (int32_t*)(b + o_c), nullptr,
                           (lpdec_stats*)(b + o_s), s);
        if (rc) { ctx->prm.lane_policy = keep; return rc; }
        CK(cudaMemcpyAsync(st.data(), b + o_s, nf * sizeof(lpdec_stats), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double t = 0.0;
        for (const auto& x : st) t += x.seconds;
        if (seconds_out) seconds_out[k] = t;
        if (t < best_t) { best_t = t; best = cand[k]; }
    }
    ctx->prm.lane_policy = best;
    if (policy_out) *policy_out = best;
    return LPDEC_OK;
}

int32_t lpdec_cut_search_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                                const double* d_u, const uint8_t* d_active, uint8_t* d_in_lp,
                                uint32_t* d_mask, int32_t* d_flag, void* stream) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 0 || (nframes > 0 && (!d_u || !d_active || !d_in_lp || !d_mask || !d_flag)))
        return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    std::lock_guard<std::mutex> g(ctx->mu);
    Launch ln;
    const bool mixed = ctx->prm.precision == LPDEC_MIXED;
    rc = mixed ? plan(ctx, code, nframes, k_cut_search<float>, 4, &ln)
               : plan(ctx, code, nframes, k_cut_search<double>, 8, &ln);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(ctx->counter, 0, sizeof(int), s));
    if (mixed)
        k_cut_search<float><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_u, d_active, d_in_lp, d_mask, d_flag, nframes,
        ctx->counter, ctx->gscratch);
    else
        k_cut_search<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_u, d_active, d_in_lp, d_mask, d_flag, nframes,
        ctx->counter, ctx->gscratch);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

int32_t lpdec_mts_select_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                                const double* d_gamma, const uint8_t* d_in_lp,
                                const uint32_t* d_mask, const double* d_w, int32_t* d_col,
                                int32_t* d_row, void* stream) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 0 || (nframes > 0 && (!d_gamma || !d_in_lp || !d_mask || !d_w || !d_col || !d_row)))
        return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    std::lock_guard<std::mutex> g(ctx->mu);
    Launch ln;
    const bool mixed = ctx->prm.precision == LPDEC_MIXED;
    rc = mixed ? plan(ctx, code, nframes, k_mts_select<float>, 4, &ln)
               : plan(ctx, code, nframes, k_mts_select<double>, 8, &ln);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(ctx->counter, 0, sizeof(int), s));
    if (mixed)
        k_mts_select<float><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_gamma, d_in_lp, d_mask, d_w, d_col, d_row,
        nframes, ctx->counter, ctx->gscratch);
    else
        k_mts_select<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_gamma, d_in_lp, d_mask, d_w, d_col, d_row,
        nframes, ctx->counter, ctx->gscratch);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

int32_t lpdec_pcg_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                         const double* d_gamma, const uint8_t* d_in_lp, const uint32_t* d_mask,
                         const double* d_d2, const double* d_w, double* d_dy, int32_t* d_iters,
                         void* stream) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 0 || (nframes > 0 && (!d_gamma || !d_in_lp || !d_mask || !d_d2 || !d_w || !d_dy || !d_iters)))
        return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    std::lock_guard<std::mutex> g(ctx->mu);
    Launch ln;
    const bool mixed = ctx->prm.precision == LPDEC_MIXED;
    rc = mixed ? plan(ctx, code, nframes, k_pcg<float>, 4, &ln)
               : plan(ctx, code, nframes, k_pcg<double>, 8, &ln);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(ctx->counter, 0, sizeof(int), s));
    if (mixed)
        k_pcg<float><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_gamma, d_in_lp, d_mask, d_d2, d_w, d_dy,
        d_iters, nframes, ctx->counter, ctx->gscratch);
    else
        k_pcg<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_gamma, d_in_lp, d_mask, d_d2, d_w, d_dy,
        d_iters, nframes, ctx->counter, ctx->gscratch);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

int32_t lpdec_pcg_trace_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                               const double* d_gamma, const uint8_t* d_in_lp,
                               const uint32_t* d_mask, const double* d_d2, const double* d_w,
                               int32_t identity, double tol, int32_t max_hist, double* d_dy,
                               int32_t* d_iters, double* d_hist, void* stream) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 0 || max_hist < 1 || !(tol > 0.0) ||
        (nframes > 0 && (!d_gamma || !d_in_lp || !d_mask || !d_d2 || !d_w || !d_dy || !d_iters ||
                         !d_hist)))
        return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    std::lock_guard<std::mutex> g(ctx->mu);
    Launch ln;
    rc = plan(ctx, code, nframes, k_pcg_trace<double>, 8, &ln);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(ctx->counter, 0, sizeof(int), s));
    k_pcg_trace<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_gamma, d_in_lp, d_mask, d_d2, d_w, d_dy,
        d_iters, d_hist, max_hist, identity ? 1 : 0, tol, nframes, ctx->counter, ctx->gscratch);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

int32_t lpdec_lp_solve_trace_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                                    const double* d_gamma, const uint8_t* d_in_lp,
                                    const uint32_t* d_mask, double* d_x, lpdec_stats* d_stats,
                                    double* d_trace, int32_t max_trace, void* stream);

int32_t lpdec_lp_solve_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                              const double* d_gamma, const uint8_t* d_in_lp,
                              const uint32_t* d_mask, double* d_x, lpdec_stats* d_stats,
                              void* stream) {
    return lpdec_lp_solve_trace_device(ctx, code, nframes, d_gamma, d_in_lp, d_mask, d_x,
                                       d_stats, nullptr, 0, stream);
}

int32_t lpdec_lp_solve_trace_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                                    const double* d_gamma, const uint8_t* d_in_lp,
                                    const uint32_t* d_mask, double* d_x, lpdec_stats* d_stats,
                                    double* d_trace, int32_t max_trace, void* stream) {
    int32_t rc = check_ctx_code(ctx, code);
    if (rc) return rc;
    if (nframes < 0 || (nframes > 0 && (!d_gamma || !d_in_lp || !d_mask || !d_x || !d_stats)))
        return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    std::lock_guard<std::mutex> g(ctx->mu);
    Launch ln;
    const bool mixed = ctx->prm.precision == LPDEC_MIXED;
    rc = mixed ? plan(ctx, code, nframes, k_lp_solve<float>, 4, &ln)
               : plan(ctx, code, nframes, k_lp_solve<double>, 8, &ln);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(ctx->counter, 0, sizeof(int), s));
    if (mixed)
        k_lp_solve<float><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_gamma, d_in_lp, d_mask, d_x, d_stats, nframes,
        ctx->counter, ctx->gscratch, d_trace, d_trace ? max_trace : 0);
    else
        k_lp_solve<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
        view_of(code, ctx->prm), to_dev(ctx->prm), ln.L, d_gamma, d_in_lp, d_mask, d_x, d_stats, nframes,
        ctx->counter, ctx->gscratch, d_trace, d_trace ? max_trace : 0);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batch decode.
//
// Some callers cannot call cudaMalloc at decode time: code that runs while
// another component owns and pre-reserves all device memory, real-time
// loops that must not enter the allocator, or hosts that forbid device
// allocation after start-up. For them, the per-CTA workspace and the frame
// queue counter of this entry point live in one file-scope device array of
// fixed size instead of in context-owned allocations. The array exists on
// every GPU that loads this library, for the life of the process.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr size_t kNoAllocCounterBytes = 256;                 // queue counter slot

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch in the current device's context. In
// host code the symbol is only a host-side stand-in; the kernel must be
// given the address returned here. It is taken on every call (no
// allocation, and no stale address after a context reset); the first call
// on a device may load the module.
int32_t noalloc_base(char** out) {
    void* ptr = nullptr;
    CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    *out = static_cast<char*>(ptr);
    return LPDEC_OK;
}

template <typename K>
int32_t noalloc_launch_plan(const lpdec_params& prm, const lpdec_code* code, int device,
                            int nframes, K kernel, size_t real_bytes, Launch* out) {
    int sms = 0, optin = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    int threads = prm.threads_per_block > 0 ? prm.threads_per_block : 128;
    threads = std::max(32, std::min(512, threads / 32 * 32));
    size_t cap = (size_t)optin - sizeof(KernelShared) - 1024;
    size_t budget = prm.smem_budget > 0 ? std::min((size_t)prm.smem_budget, cap) : cap;
    Dims d;
    d.cover(view_of(code, prm));
    const size_t avail = kNoAllocScratchBytes - kNoAllocCounterBytes;
    // The dense fallback of stalled Newton solves, as in the regular entry,
    // whenever one CTA's workspace with its matrix fits the array; the grid
    // then shrinks to the CTAs the array holds.
    const bool m32 = prm.precision == LPDEC_M32;
    Layout L, Lw;
    bool ok = make_layouts(d, budget, real_bytes, m32, dense_rows_for(d), &L, &Lw);
    if (ok && L.stride > avail) ok = make_layouts(d, budget, real_bytes, m32, 0, &L, &Lw);
    if (!ok || L.smem_bytes + sizeof(KernelShared) > (size_t)optin) {
        snprintf(g_err, sizeof g_err, "frame workspace does not fit in shared memory");
        return LPDEC_ERR_INVALID_ARG;
    }
    if (L.stride > avail) {
        snprintf(g_err, sizeof g_err,
                 "one frame needs %llu bytes of scratch, above the %zu-byte static array",
                 (unsigned long long)L.stride, avail);
        return LPDEC_ERR_OUT_OF_BUDGET;
    }
    CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, L.smem_bytes));
    if (per_sm < 1) {
        snprintf(g_err, sizeof g_err, "kernel does not fit on an SM");
        return LPDEC_ERR_INVALID_ARG;
    }
    size_t by_scratch = L.stride ? avail / L.stride : (size_t)per_sm * sms;
    int grid = (int)std::min<size_t>({(size_t)nframes, (size_t)per_sm * sms, by_scratch});
    out->L = L;
    out->Lw = Lw;
    out->threads = threads;
    out->grid = std::max(1, grid);
    return LPDEC_OK;
}

}  // namespace

extern "C" int32_t lpdec_decode_batch_device_noalloc(const lpdec_code* code,
                                                     const lpdec_params* params,
                                                     int32_t nframes, const double* d_gamma,
                                                     double* d_u, uint8_t* d_hard,
                                                     int32_t* d_cert, uint32_t* d_cut_mask,
                                                     lpdec_stats* d_stats, void* stream) {
    if (!code || !code->ctx || nframes < 0 ||
        (nframes > 0 && (!d_gamma || !d_u || !d_hard || !d_cert)))
        return LPDEC_ERR_INVALID_ARG;
    lpdec_params prm;
    if (params) prm = *params; else lpdec_default_params(&prm);
    if (!params_ok(prm)) return LPDEC_ERR_INVALID_ARG;
    if (nframes == 0) return LPDEC_OK;
    const int device = code->device;
    CK(cudaSetDevice(device));
    char* base = nullptr;
    int32_t rc = noalloc_base(&base);
    if (rc) return rc;
    const bool mixed = prm.precision == LPDEC_MIXED;
    Launch ln;
    rc = mixed ? noalloc_launch_plan(prm, code, device, nframes, k_decode<float>, 4, &ln)
               : noalloc_launch_plan(prm, code, device, nframes, k_decode<double>, 8, &ln);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int* counter = reinterpret_cast<int*>(base);
    char* gscratch = base + kNoAllocCounterBytes;
    CK(cudaMemsetAsync(counter, 0, sizeof(int), s));   // the only state a call must reset
    if (mixed)
        k_decode<float><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
            view_of(code, prm), nullptr, nullptr, to_dev(prm), ln.L, ln.Lw, d_gamma, d_u, d_hard,
            d_cert, d_cut_mask, d_stats,
            nframes, counter, gscratch, nullptr);
    else
        k_decode<double><<<ln.grid, ln.threads, ln.L.smem_bytes, s>>>(
            view_of(code, prm), nullptr, nullptr, to_dev(prm), ln.L, ln.Lw, d_gamma, d_u, d_hard,
            d_cert, d_cut_mask, d_stats,
            nframes, counter, gscratch, nullptr);
    CK(cudaGetLastError());
    return LPDEC_OK;
}

#include "serve.cuh"
