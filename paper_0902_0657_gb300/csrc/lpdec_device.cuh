// Device side of the adaptive LP decoder: every step of the hot path as
// CTA-cooperative device functions. One CTA decodes one frame. The arrays
// touched inside the PCG loop (packed LP structure, level schedules, PCG
// vectors) live in shared memory; the interior-point state (FP64 x, y, z,
// ...) lives in per-CTA global scratch, which stays resident in L2.
//
// Paper: Taghavi, Shokrollahi, Siegel, "Efficient Implementation of Linear
// Programming Decoding". Section/equation/algorithm numbers below refer to
// it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lpdec.h"

namespace lpdec {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint8_t kInLP = 1;     // check j has at least one parity inequality in the LP
constexpr uint8_t kActive = 2;   // ... and one of them is active at the last LP solution
constexpr uint8_t kNew = 4;      // the cut search found a violated inequality of j this round
constexpr uint16_t kNone = 0xffffu;
constexpr uint16_t kNeg = 0x8000u;   // packed entry: index | kNeg if the coefficient is -1
constexpr uint16_t kIdx = 0x7fffu;

// ---------------------------------------------------------------------------
// Code (H) view: CSR rows = checks, CSC columns = bits. Read-only, shared by
// every frame of the code (n, m <= 32767). pmax / eamax: capacity of one
// frame's LP (rows, and nonzeros of the standard part of A) in the main
// workspace; pwide / eawide: in the wide workspace a frame moves to when its
// cut list outgrows the main one (ALP holds several rows per check).
// ---------------------------------------------------------------------------
struct CodeView {
    int n, m, E;
    int pmax, eamax, pwide, eawide;
    const int* __restrict__ h_ptr;   // [m+1]
    const int* __restrict__ h_col;   // [E] bit of CSR edge e
    const int* __restrict__ e_chk;   // [E] check of CSR edge e
    const int* __restrict__ v_ptr;   // [n+1]
    const int* __restrict__ v_chk;   // [E] check of the k-th CSC entry
    const int* __restrict__ v_eidx;  // [E] CSR edge index of the k-th CSC entry
};

struct DevParams {
    double sigma, eta, tol_gap, tol_feas, tol_pcg, tau_act, tau_cut, tau_int;
    double pcg_gap_factor, tol_inner, tol_feas_loose, tol_cert, tau_inc;
    int max_alp, max_ipm, max_pcg, variant, precision;
    int precond, precond_switch;
    int warm_start, mts_reuse;
    int lane_policy;
    int dense_switch;
    // serving: the frame's cancel flag in mapped host memory (null outside
    // the server); read by thread 0 between LPs and every 4th IPM iteration
    const volatile int32_t* abort;
};

// Whether the frame's cancel flag is set (the same value in every thread).
__device__ __forceinline__ bool aborted(const DevParams& P) {
    int a = 0;
    if (P.abort && threadIdx.x == 0) a = *P.abort != 0;
    return __syncthreads_or(a) != 0;
}

// ---------------------------------------------------------------------------
// Workspace layout (the host decides shared vs global placement). Arrays over
// LP rows have the capacity pmax, arrays over columns n + pmax.
// ---------------------------------------------------------------------------
enum Arr {
    // LP structure: cut list (rows grouped by check), packed row entries and
    // column entries of A, per-check row pointers
    S_ROWENT, S_COLENT, S_CCHK, S_CMASK, S_CACT, S_RPTR, S_CPTR, S_CRPTR,
    // preconditioner selection and the two level-scheduled triangular solves
    S_PIVCOL, S_PIVROW, S_PSGN,
    S_LB, S_LF, S_LBPTR, S_LFPTR, S_CUR, S_LBROWS, S_LFROWS, S_SELROW,
    S_DEG, S_BITMAP, S_FLAGS, S_MASK, S_FLIP, S_HPTR, S_VPTR,
    S_BPTR, S_BDEP, S_FPTR, S_FDEP,   // dependency lists of the two triangular solves
    S_LBSE, S_LFSE,   // per level position: the dependency range of its row (sweep order)
    S_VEC,      // PCG vectors the triangular sweeps read on their serial path, type T:
                // r, z, invd2p (pmax each) [+ 3 FP32 vectors, LPDEC_M32]; during the
                // MTS selection the same bytes hold rank [q] and sorted [q]
    S_VECC,     // PCG vectors only the parallel passes touch, type T: xs, h, l (pmax
                // each), t (n), d2t (n+pmax); during the MTS selection the same bytes
                // hold the sort keys (u64 [q2], u32 [q2])
    // FP64 interior-point state (global scratch)
    G_X, G_Z, G_RC, G_D2, G_Y, G_B, G_W, G_DY, G_R64, G_U, G_T64, G_BASIC,
    // optimality certificate scratch: vertex and CG vectors over columns
    // (4 x n+pmax) and rows (2 x pmax)
    G_VX, G_V1, G_V2, G_V3, G_V4, G_VR1, G_VR2,
    // FP64 PCG vectors for the fallback rounds of the mixed mode (xs, r, z,
    // h, l, t, invd2p)
    G_P64,
    // dense p x p FP64 matrix of the Cholesky fallback of the Newton solve
    // (16 bytes when the fallback is off)
    G_QD,
    // cut list being rebuilt (rows, masks, per-check row pointers) after a cut search
    G_CCHK2, G_CMASK2, G_CRPTR2,
    // the CTA's copy of the frame's LLRs (serving: read from the shared arena
    // once, past the SM's L1)
    G_GAM,
    // CG coefficients of the first PCG round of a traced Newton solve
    G_LZ,
    // warm start: the previous LP's final iterate (x, z over its columns, y
    // over its rows) and, per check, its row there and that row's set V
    G_XW, G_ZW, G_YW, G_PROW, G_PMASK,
    A_COUNT
};

constexpr uint32_t kGlobalBit = 0x80000000u;

// FP64 elements of the G_P64 block (xs, r, z, h, l, t, invd2p) with room
// for d2t (n + pmax): 7 pmax + 2n.
__host__ __device__ constexpr size_t vec_elems(int n, int pmax) {
    return 7 * (size_t)pmax + 2 * (size_t)n;
}
// Bytes of the S_VEC block: r, z, invd2p in type T and, for LPDEC_M32,
// three FP32 vectors after them (the M-solve's right side and solution, and
// 1/d^2 of the pivot columns); at least rank and sorted.
__host__ __device__ constexpr size_t vec_hot_bytes(int n, int pmax, size_t real_bytes, bool m32) {
    return (real_bytes * 3 * (size_t)pmax + (m32 ? 12 * (size_t)pmax : 0)) >
                   4 * ((size_t)n + pmax)
               ? real_bytes * 3 * (size_t)pmax + (m32 ? 12 * (size_t)pmax : 0)
               : 4 * ((size_t)n + pmax);
}
// Bytes of the S_VECC block: xs, h, l, t, d2t in type T, at least the sort
// keys.
__host__ __device__ constexpr size_t vec_cold_bytes(int n, int pmax, size_t real_bytes,
                                                    size_t q2) {
    return real_bytes * (2 * (size_t)n + 4 * (size_t)pmax) > 12 * q2
               ? real_bytes * (2 * (size_t)n + 4 * (size_t)pmax)
               : 12 * q2;
}

struct Layout {
    uint32_t off[A_COUNT];     // byte offset; kGlobalBit set = global scratch
    uint32_t smem_bytes;       // dynamic shared memory per CTA
    uint32_t q2;               // power of two >= nmax + pmax (sort width)
    uint32_t dense;            // rows of the dense fallback's FP64 matrix in G_QD (0: off)
    uint32_t nmax, mmax, pmax; // capacities the arrays are sized for
    unsigned long long gbytes; // global scratch bytes of this workspace per CTA
    unsigned long long stride; // global scratch bytes per CTA (main + wide workspace)
};

// Arrays whose size depends on the LP's row capacity; a frame moved to the
// wide workspace takes these from it and keeps the others (per check, per
// bit, the code's pointers, the dense fallback's matrix) where they were.
__host__ __device__ constexpr bool row_sized(int a) {
    return !(a == S_FLAGS || a == S_MASK || a == S_FLIP || a == S_HPTR || a == S_VPTR ||
             a == S_CPTR || a == S_CRPTR || a == G_U || a == G_T64 || a == G_QD ||
             a == G_CRPTR2 || a == G_GAM || a == G_LZ || a == G_PROW || a == G_PMASK);
}

template <typename T>
struct WS {
    uint16_t *rowent, *colent, *cchk, *pivcol, *pivrow, *lb, *lf, *lbrows, *lfrows;
    uint16_t *selrow, *rank, *sorted, *deg;
    uint32_t *cmask, *rptr, *cptr, *crptr;
    uint32_t *lbptr, *lfptr, *cur, *bitmap, *mask, *flip;
    int *hptr, *vptr;   // shared copies of the code's CSR / CSC row pointers
    uint32_t *bptr, *fptr;
    uint16_t *bdep, *fdep;   // packed (row | kNeg): rows whose solved values row r needs
    uint2 *lbse, *lfse;      // dependency range (begin, end) of the row at each level position
    uint8_t *cact, *psgn, *flags, *basic;
    T *xs, *r, *z, *h, *l, *t, *d2t, *invd2p;
    float *rf, *zf, *ip32;      // FP32 M-solve vectors (LPDEC_M32 only)
    unsigned long long* skey;   // aliases the PCG vectors
    uint32_t* sidx;             // column index of each sort key
    double *x, *zz, *rc, *d2, *y, *b, *w, *dy, *r64, *u, *t64;
    double *vx, *v1, *v2, *v3, *v4, *vr1, *vr2, *p64;
    double* qd;   // dense Cholesky factor (column-major p x p), null when off
    double* gam;  // private copy of the frame's LLRs (serving)
    double* lz;   // CG coefficient record of traced solves (null when not tracing)
    double *xw, *zw, *yw;   // warm start: previous LP's final iterate
    int* prow;              // ... per check: its row in the previous LP (-1: none)
    uint32_t* pmask;        // ... and that row's set V
    uint16_t* cchk2;
    uint32_t *cmask2, *crptr2;
    int cap_n, cap_p;   // capacities the sub-arrays were sliced with
    int lanes;          // lanes per row of the warp-mode sweeps (0: by level width)
    int dense_p;        // rows the dense fallback's matrix holds (0: off)
};

__device__ __forceinline__ char* ws_ptr(const Layout& L, int a, char* smem, char* gws) {
    uint32_t o = L.off[a];
    return (o & kGlobalBit) ? gws + (o & ~kGlobalBit) : smem + o;
}

// Pointers of one CTA's workspace; sub-arrays of S_VEC and G_P64 are sliced
// with the layout's capacities, so frames of any smaller code fit. With
// only_rows, only the row-sized arrays are (re)pointed (moving a frame to the
// wide workspace).
template <typename T>
__device__ inline void point_ws(WS<T>& w, const Layout& L, char* smem, char* gws, bool only_rows) {
    const int n = (int)L.nmax, pm = (int)L.pmax;
#define P_(Ty, name, id) \
    if (!only_rows || row_sized(id)) w.name = reinterpret_cast<Ty*>(ws_ptr(L, id, smem, gws))
    P_(uint16_t, rowent, S_ROWENT); P_(uint16_t, colent, S_COLENT);
    P_(uint16_t, cchk, S_CCHK); P_(uint32_t, cmask, S_CMASK); P_(uint8_t, cact, S_CACT);
    P_(uint32_t, rptr, S_RPTR); P_(uint32_t, cptr, S_CPTR); P_(uint32_t, crptr, S_CRPTR);
    P_(uint16_t, pivcol, S_PIVCOL); P_(uint16_t, pivrow, S_PIVROW);
    P_(uint8_t, psgn, S_PSGN);
    P_(uint16_t, lb, S_LB); P_(uint16_t, lf, S_LF);
    P_(uint32_t, lbptr, S_LBPTR); P_(uint32_t, lfptr, S_LFPTR); P_(uint32_t, cur, S_CUR);
    P_(uint16_t, lbrows, S_LBROWS); P_(uint16_t, lfrows, S_LFROWS); P_(uint16_t, selrow, S_SELROW);
    P_(uint16_t, deg, S_DEG);
    P_(uint32_t, bitmap, S_BITMAP); P_(uint8_t, flags, S_FLAGS); P_(uint32_t, mask, S_MASK);
    P_(uint32_t, flip, S_FLIP);
    P_(int, hptr, S_HPTR); P_(int, vptr, S_VPTR);
    P_(uint32_t, bptr, S_BPTR); P_(uint32_t, fptr, S_FPTR);
    P_(uint16_t, bdep, S_BDEP); P_(uint16_t, fdep, S_FDEP);
    P_(uint2, lbse, S_LBSE); P_(uint2, lfse, S_LFSE);
    if (!only_rows || row_sized(S_VEC)) {
        T* v = reinterpret_cast<T*>(ws_ptr(L, S_VEC, smem, gws));
        w.rank = reinterpret_cast<uint16_t*>(v);
        w.sorted = w.rank + (n + pm);
        w.r = v; v += pm; w.z = v; v += pm; w.invd2p = v;
        w.rf = reinterpret_cast<float*>(w.invd2p + pm); w.zf = w.rf + pm; w.ip32 = w.zf + pm;
        T* c = reinterpret_cast<T*>(ws_ptr(L, S_VECC, smem, gws));
        w.skey = reinterpret_cast<unsigned long long*>(c);
        w.sidx = reinterpret_cast<uint32_t*>(w.skey + L.q2);
        w.xs = c; c += pm; w.h = c; c += pm; w.l = c; c += pm;
        w.t = c; c += n; w.d2t = c;
    }
    P_(double, x, G_X); P_(double, zz, G_Z); P_(double, rc, G_RC); P_(double, d2, G_D2);
    P_(double, y, G_Y); P_(double, b, G_B); P_(double, w, G_W); P_(double, dy, G_DY);
    P_(double, r64, G_R64); P_(double, u, G_U); P_(double, t64, G_T64);
    P_(uint8_t, basic, G_BASIC);
    P_(double, vx, G_VX); P_(double, v1, G_V1); P_(double, v2, G_V2); P_(double, v3, G_V3);
    P_(double, v4, G_V4); P_(double, vr1, G_VR1); P_(double, vr2, G_VR2);
    P_(double, p64, G_P64);
    P_(double, qd, G_QD);
    P_(uint16_t, cchk2, G_CCHK2); P_(uint32_t, cmask2, G_CMASK2);
    P_(uint32_t, crptr2, G_CRPTR2);
    P_(double, gam, G_GAM);
    P_(double, lz, G_LZ);
    P_(double, xw, G_XW); P_(double, zw, G_ZW); P_(double, yw, G_YW);
    P_(int, prow, G_PROW); P_(uint32_t, pmask, G_PMASK);
#undef P_
    if (!only_rows) w.lz = nullptr;   // set by the traced entry point only
    if (!only_rows) {
        if (!L.dense) w.qd = nullptr;
        w.dense_p = (int)L.dense;
    }
    w.cap_n = n;
    w.cap_p = pm;
    if (!only_rows) w.lanes = 0;
}

template <typename T>
__device__ inline WS<T> make_ws(const Layout& L, char* smem, char* gws) {
    WS<T> w;
    point_ws<T>(w, L, smem, gws, false);
    return w;
}

// A view with FP64 PCG vectors (in global scratch) and the same LP
// structure, for the FP64 fallback rounds of the mixed mode. d2t is the FP64
// D^2 itself.
template <typename T>
__device__ inline WS<double> fp64_view(const WS<T>& W) {
    const int n = W.cap_n, pm = W.cap_p;
    WS<double> v;
    v.cap_n = n;
    v.cap_p = pm;
    v.dense_p = W.dense_p;
    v.lanes = W.lanes;
    v.rowent = W.rowent; v.colent = W.colent; v.cchk = W.cchk; v.cmask = W.cmask;
    v.cact = W.cact; v.rptr = W.rptr; v.cptr = W.cptr; v.crptr = W.crptr;
    v.pivcol = W.pivcol; v.pivrow = W.pivrow; v.lb = W.lb; v.lf = W.lf; v.lbrows = W.lbrows;
    v.lfrows = W.lfrows; v.selrow = W.selrow; v.rank = W.rank; v.sorted = W.sorted;
    v.lbptr = W.lbptr; v.lfptr = W.lfptr; v.cur = W.cur; v.bitmap = W.bitmap; v.mask = W.mask;
    v.flip = W.flip; v.psgn = W.psgn; v.deg = W.deg; v.flags = W.flags; v.basic = W.basic;
    v.hptr = W.hptr; v.vptr = W.vptr;
    v.bptr = W.bptr; v.fptr = W.fptr; v.bdep = W.bdep; v.fdep = W.fdep;
    v.lbse = W.lbse; v.lfse = W.lfse;
    double* q = W.p64;
    v.xs = q; q += pm; v.r = q; q += pm; v.z = q; q += pm; v.h = q; q += pm; v.l = q; q += pm;
    v.t = q; q += n; v.invd2p = q;
    v.rf = W.rf; v.zf = W.zf; v.ip32 = W.ip32;
    v.d2t = W.d2;
    v.skey = nullptr;
    v.sidx = nullptr;
    v.x = W.x; v.zz = W.zz; v.rc = W.rc; v.d2 = W.d2; v.y = W.y; v.b = W.b; v.w = W.w;
    v.dy = W.dy; v.r64 = W.r64; v.u = W.u; v.t64 = W.t64;
    v.vx = W.vx; v.v1 = W.v1; v.v2 = W.v2; v.v3 = W.v3; v.v4 = W.v4; v.vr1 = W.vr1;
    v.vr2 = W.vr2; v.p64 = W.p64; v.qd = W.qd; v.gam = W.gam; v.lz = W.lz;
    v.xw = W.xw; v.zw = W.zw; v.yw = W.yw; v.prow = W.prow; v.pmask = W.pmask;
    v.cchk2 = W.cchk2; v.cmask2 = W.cmask2; v.crptr2 = W.crptr2;
    return v;
}

// Copies the code's row and column pointers into the workspace (shared
// memory) and returns a view of the code that reads them from there.
template <typename T>
__device__ inline CodeView bind_code(const CodeView& C, WS<T>& W) {
    __syncthreads();   // the previous frame may still read the old pointers
    for (int k = threadIdx.x; k <= C.m; k += blockDim.x) W.hptr[k] = C.h_ptr[k];
    for (int k = threadIdx.x; k <= C.n; k += blockDim.x) W.vptr[k] = C.v_ptr[k];
    __syncthreads();
    CodeView v = C;
    v.h_ptr = W.hptr;
    v.v_ptr = W.vptr;
    return v;
}

// ---------------------------------------------------------------------------
// Block helpers
// ---------------------------------------------------------------------------
struct Blk {
    int tid, nt, lane, warp, nwarps;
    double* red;   // shared [2][64]
    int phase;
    int sw;        // the warp that runs the CTA's single-warp phases (level
                   // sweeps, MTS greedy); rotated over the CTAs of an SM so
                   // that their serial chains use different SM sub-partitions
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return __shfl_sync(kFull, v, 0);
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Sums of a and b over the block; every thread gets the same values (fixed
// association order: warp tree, then warps in index order).
__device__ inline double2 bsum2(Blk& B, double a, double b) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(kFull, a, o);
        b += __shfl_down_sync(kFull, b, o);
    }
    double* buf = B.red + (B.phase & 1) * 64;
    if (B.lane == 0) { buf[B.warp] = a; buf[32 + B.warp] = b; }
    __syncthreads();
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < B.nwarps; ++k) { sa += buf[k]; sb += buf[32 + k]; }
    B.phase++;
    return make_double2(sa, sb);
}
__device__ inline double bsum(Blk& B, double a) { return bsum2(B, a, 0.0).x; }

__device__ inline double2 bmin2(Blk& B, double a, double b) {
    for (int o = 16; o > 0; o >>= 1) {
        a = fmin(a, __shfl_down_sync(kFull, a, o));
        b = fmin(b, __shfl_down_sync(kFull, b, o));
    }
    double* buf = B.red + (B.phase & 1) * 64;
    if (B.lane == 0) { buf[B.warp] = a; buf[32 + B.warp] = b; }
    __syncthreads();
    double sa = INFINITY, sb = INFINITY;
    for (int k = 0; k < B.nwarps; ++k) { sa = fmin(sa, buf[k]); sb = fmin(sb, buf[32 + k]); }
    B.phase++;
    return make_double2(sa, sb);
}

// Exclusive prefix sum of one int per thread over the block.
__device__ inline int bscan_excl(Blk& B, int v, int* total, int* sh /*[33]*/) {
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (B.lane >= o) x += y;
    }
    if (B.lane == 31) sh[B.warp] = x;
    __syncthreads();
    if (B.warp == 0) {
        int s = (B.lane < B.nwarps) ? sh[B.lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, s, o);
            if (B.lane >= o) s += y;
        }
        if (B.lane < B.nwarps) sh[B.lane] = s;   // inclusive warp totals
    }
    __syncthreads();
    int base = (B.warp > 0) ? sh[B.warp - 1] : 0;
    *total = sh[B.nwarps - 1];
    __syncthreads();
    return base + x - v;
}

__device__ __forceinline__ bool flipped(const uint32_t* fl, int i) {
    return (fl[i >> 5] >> (i & 31)) & 1u;
}
template <typename T>
__device__ __forceinline__ T signed_val(uint16_t ent, T v) { return (ent & kNeg) ? -v : v; }

// ---------------------------------------------------------------------------
// Frame state
// ---------------------------------------------------------------------------
// Device global timer (ns); the phase times of lpdec_stats.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ double since(unsigned long long t0) {
    return 1e-9 * (double)(global_ns() - t0);
}

struct Frame {
    int p;          // LP rows
    int q;          // n + p
    double normb, normc;
    int ea;         // nonzeros of the standard part of A (sum of the LP rows' degrees)
};

// u^0 = bitwise hard decision (Eq. 8); empty cut list.
template <typename T>
__device__ inline void frame_init(Blk& B, const CodeView& C, WS<T>& W, const double* gamma) {
    for (int i = B.tid; i < C.n; i += B.nt) W.u[i] = gamma[i] < 0.0 ? 1.0 : 0.0;
    for (int k = B.tid; k < (C.n + 31) / 32; k += B.nt) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            int i = k * 32 + b;
            if (i < C.n && gamma[i] < 0.0) bits |= 1u << b;
        }
        W.flip[k] = bits;
    }
    for (int j = B.tid; j < C.m; j += B.nt) { W.flags[j] = 0; W.mask[j] = 0; }
    for (int j = B.tid; j <= C.m; j += B.nt) W.crptr[j] = 0;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// a1: cut search — Algorithm 2 per check inside the loop of Algorithm 3 (or
// Algorithm 1). One warp per check, lanes = neighbours (d_j <= 32). MALP
// searches the checks without an active inequality; ALP searches every
// check. A violated check gets kNew and its set V in mask[j].
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline int cut_search(Blk& B, const CodeView& C, WS<T>& W, const DevParams& P,
                                 bool alp) {
    int added = 0;
    for (int j = B.warp; j < C.m; j += B.nwarps) {
        uint8_t f = W.flags[j];
        if (!alp && (f & kInLP) && (f & kActive)) continue;   // j has an active inequality
        int beg = C.h_ptr[j];
        int d = C.h_ptr[j + 1] - beg;
        if (d <= 0) continue;
        bool valid = B.lane < d;
        double ui = valid ? W.u[C.h_col[beg + B.lane]] : 0.0;
        unsigned S = __ballot_sync(kFull, valid && ui > 0.5);     // S = {u_i > 1/2}
        unsigned V = S;
        if ((__popc(S) & 1) == 0) {                                // |S| even
            double dist = valid ? fabs(ui - 0.5) : INFINITY;
            double mn = warp_min(dist);
            unsigned tie = __ballot_sync(kFull, valid && dist == mn);
            V ^= 1u << (__ffs(tie) - 1);                           // toggle i* (lowest on ties)
        }
        double term = valid ? (((V >> B.lane) & 1u) ? 1.0 - ui : ui) : 0.0;
        double lhs = warp_sum(term);                               // left side of Eq. 6
        if (lhs < 1.0 - P.tau_cut) {
            if (B.lane == 0) { W.mask[j] = V; W.flags[j] = f | kInLP | kNew; }
            added = 1;
        }
    }
    return __syncthreads_or(added);
}

// MALP-B: drop every inactive inequality before the search (Section III-A).
template <typename T>
__device__ inline void drop_inactive(Blk& B, const CodeView& C, WS<T>& W) {
    for (int j = B.tid; j < C.m; j += B.nt) {
        uint8_t f = W.flags[j];
        if ((f & kInLP) && !(f & kActive)) { W.flags[j] = 0; W.mask[j] = 0; }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// a2: augmented LP (Eq. 16) from the cut list. A row r is a cut (check
// cchk[r], odd set cmask[r]); rows are grouped by check (crptr[j] .. crptr[j+1])
// and ordered by insertion inside a check. Rebuilding the list after a cut
// search keeps a check's old rows unless it is not in the LP any more or
// (MALP, alp = false) its new cut replaces them, and appends the new cut.
// Coefficients are +-1: a_{r,i} = s_i (unflipped) or -s_i (flipped),
// s_i = +1 iff i in V, and b_r = |V| - 1 - sum_{flipped i in N(j)} s_i.
// Packed entries: rowent[rptr[r] + t] = bit | sign of the t-th neighbour of
// the row's check; colent[cptr[i] ..] = (row | sign) over the rows that hold
// bit i, in increasing row order. Returns false (LP left unchanged) when the
// new list exceeds the workspace's capacity (pcap rows, eacap entries).
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline bool lp_build(Blk& B, const CodeView& C, WS<T>& W, Frame& F, int* shscan,
                                bool alp, int pcap, int eacap) {
    // 1. new cut list, grouped by check
    int per = (C.m + B.nt - 1) / B.nt;
    int j0 = B.tid * per, j1 = min(C.m, j0 + per);
    int cnt = 0, cne = 0;
    for (int j = j0; j < j1; ++j) {
        uint8_t f = W.flags[j];
        int kept = ((f & kInLP) && !(!alp && (f & kNew))) ? (int)(W.crptr[j + 1] - W.crptr[j]) : 0;
        int c = kept + ((f & kNew) ? 1 : 0);
        cnt += c;
        cne += c * (C.h_ptr[j + 1] - C.h_ptr[j]);
    }
    int p, ne_all;
    int pos = bscan_excl(B, cnt, &p, shscan);
    bscan_excl(B, cne, &ne_all, shscan);
    if (p > pcap || ne_all > eacap) return false;   // same decision in every thread
    // (the old list is only read until the barrier; the new one goes to the
    // G_*2 arrays first)
    for (int j = j0; j < j1; ++j) {
        uint8_t f = W.flags[j];
        W.crptr2[j] = (uint32_t)pos;
        if ((f & kInLP) && !(!alp && (f & kNew)))
            for (uint32_t r = W.crptr[j]; r < W.crptr[j + 1]; ++r) {
                W.cchk2[pos] = (uint16_t)j;
                W.cmask2[pos] = W.cmask[r];
                ++pos;
            }
        if (f & kNew) { W.cchk2[pos] = (uint16_t)j; W.cmask2[pos] = W.mask[j]; ++pos; }
    }
    if (B.tid == 0) W.crptr2[C.m] = (uint32_t)p;
    __syncthreads();
    for (int j = B.tid; j <= C.m; j += B.nt) {
        const uint32_t a = W.crptr2[j];
        W.crptr[j] = a;
        // kNew consumed; activity is set by the next LP
        if (j < C.m) W.flags[j] = (W.crptr2[j + 1] > a) ? kInLP : 0;
    }
    for (int r = B.tid; r < p; r += B.nt) { W.cchk[r] = W.cchk2[r]; W.cmask[r] = W.cmask2[r]; }
    __syncthreads();
    // 2. row pointers (row r holds d_j entries)
    per = (p + B.nt - 1) / B.nt;
    const int r0 = B.tid * per, r1 = min(p, r0 + per);
    int ne = 0;
    for (int r = r0; r < r1; ++r) { int j = W.cchk[r]; ne += C.h_ptr[j + 1] - C.h_ptr[j]; }
    int ea;
    int epos = bscan_excl(B, ne, &ea, shscan);
    for (int r = r0; r < r1; ++r) {
        W.rptr[r] = (uint32_t)epos;
        int j = W.cchk[r];
        epos += C.h_ptr[j + 1] - C.h_ptr[j];
    }
    if (B.tid == 0) W.rptr[p] = (uint32_t)ea;
    __syncthreads();
    // 3. row entries and b
    double nb2 = 0.0;
    for (int r = B.tid; r < p; r += B.nt) {
        const int j = W.cchk[r], beg = C.h_ptr[j], d = C.h_ptr[j + 1] - beg;
        const uint32_t V = W.cmask[r];
        const uint32_t o = W.rptr[r];
        double shift = 0.0;
        for (int t = 0; t < d; ++t) {
            const int i = C.h_col[beg + t];
            const bool inV = (V >> t) & 1u;
            const bool fl = flipped(W.flip, i);
            W.rowent[o + t] = (uint16_t)(i | ((inV == fl) ? kNeg : 0));
            if (fl) shift += inV ? 1.0 : -1.0;
        }
        double bv = (double)__popc(V) - 1.0 - shift;
        W.b[r] = bv;
        nb2 += bv * bv;
    }
    // 4. column pointers and entries (rows of bit i: the rows of its checks)
    per = (C.n + B.nt - 1) / B.nt;
    const int i0 = B.tid * per, i1 = min(C.n, i0 + per);
    int nc = 0;
    for (int i = i0; i < i1; ++i)
        for (int k = C.v_ptr[i]; k < C.v_ptr[i + 1]; ++k) {
            int j = C.v_chk[k];
            nc += (int)(W.crptr[j + 1] - W.crptr[j]);
        }
    int tot;
    int cpos = bscan_excl(B, nc, &tot, shscan);   // barrier inside: rowent complete
    for (int i = i0; i < i1; ++i) {
        W.cptr[i] = (uint32_t)cpos;
        for (int k = C.v_ptr[i]; k < C.v_ptr[i + 1]; ++k) {
            const int j = C.v_chk[k];
            const int t = C.v_eidx[k] - C.h_ptr[j];
            for (uint32_t r = W.crptr[j]; r < W.crptr[j + 1]; ++r)
                W.colent[cpos++] = (uint16_t)(r | (W.rowent[W.rptr[r] + t] & kNeg));
        }
    }
    if (B.tid == 0) W.cptr[C.n] = (uint32_t)tot;
    F.p = p;
    F.q = C.n + p;
    F.ea = ea;
    F.normb = sqrt(bsum(B, nb2));   // (barrier inside)
    return true;
}

// (A' v)_i for a standard column i (its LP rows, through colent).
template <typename V, typename T>
__device__ __forceinline__ V colA_T(const CodeView& C, const WS<T>& W, int i, const V* v) {
    V acc = V(0);
    const uint32_t k1 = W.cptr[i + 1];
    for (uint32_t k = W.cptr[i]; k < k1; ++k) {
        uint16_t ent = W.colent[k];
        acc += signed_val<V>(ent, v[ent & kIdx]);
    }
    return acc;
}
// (A v)_r over the standard part of LP row r (slack added by the caller).
template <typename V, typename T>
__device__ __forceinline__ V rowA(const CodeView& C, const WS<T>& W, int r, const V* vq) {
    V acc = V(0);
    const uint32_t e1 = W.rptr[r + 1];
    for (uint32_t e = W.rptr[r]; e < e1; ++e) {
        uint16_t ent = W.rowent[e];
        acc += signed_val<V>(ent, vq[ent & kIdx]);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// a4: column-wise greedy MTS (Algorithm 7) with weights wt[0..q).
// Columns are ranked once by (weight desc, index asc) with a bitonic sort on
// the FP64 weights; DEG1 is a bitmap over ranks, so "maximum-weight
// degree-1 column" is the first set bit. One warp runs the p greedy steps:
// lanes scan the bitmap and update the columns of the removed row. The
// forward-solve level of each row is fixed when its pivot is chosen and the
// back-substitution levels follow in reverse selection order.
// ---------------------------------------------------------------------------

// Bitonic sort of n2 (a power of two) composite keys (key, idx), ascending.
__device__ inline void bitonic_sort(Blk& B, unsigned long long* key, uint32_t* idx, int n2) {
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = B.tid; t < (n2 >> 1); t += B.nt) {
                int i = 2 * t - (t & (j - 1));
                int l = i + j;
                bool up = (i & k) == 0;
                unsigned long long ki = key[i], kl = key[l];
                uint32_t ii = idx[i], il = idx[l];
                bool gt = ki > kl || (ki == kl && ii > il);
                if (gt == up) { key[i] = kl; key[l] = ki; idx[i] = il; idx[l] = ii; }
            }
            __syncthreads();
        }
    }
}

struct Levels { int nb, nf; };

// Dependency lists of the two triangular solves, in CSR form over the LP
// rows: row r's back-substitution step needs the solved values of the rows
// pivoting the other selected columns of row r; its forward step needs the
// other rows of its own pivot column. Each entry is (row | kNeg when the
// coefficient is -1).
template <typename T>
__device__ inline void build_deps(Blk& B, const CodeView& C, WS<T>& W, const Frame& F) {
    const int n = C.n, p = F.p;
    int* sh = reinterpret_cast<int*>(B.red);   // scan scratch (33 ints) in the reduction buffer
    const int per = (p + B.nt - 1) / B.nt;
    const int r0 = B.tid * per, r1 = min(p, r0 + per);
    int cb = 0, cf = 0;
    for (int r = r0; r < r1; ++r) {
        const int i0 = W.pivcol[r];
        for (uint32_t e = W.rptr[r]; e < W.rptr[r + 1]; ++e) {
            int i2 = W.rowent[e] & kIdx;
            cb += (i2 != i0 && W.pivrow[i2] != kNone);
        }
        if (i0 < n) cf += (int)(W.cptr[i0 + 1] - W.cptr[i0]) - 1;
    }
    int tb, tf;
    int ob = bscan_excl(B, cb, &tb, sh);
    int of = bscan_excl(B, cf, &tf, sh);
    for (int r = r0; r < r1; ++r) {
        const int i0 = W.pivcol[r];
        W.bptr[r] = ob;
        W.fptr[r] = of;
        for (uint32_t e = W.rptr[r]; e < W.rptr[r + 1]; ++e) {
            uint16_t ent = W.rowent[e];
            int i2 = ent & kIdx;
            if (i2 == i0) continue;
            uint16_t pr = W.pivrow[i2];
            if (pr != kNone) W.bdep[ob++] = (uint16_t)(pr | (ent & kNeg));
        }
        if (i0 < n)
            for (uint32_t k = W.cptr[i0]; k < W.cptr[i0 + 1]; ++k) {
                uint16_t ent = W.colent[k];
                if ((ent & kIdx) != r) W.fdep[of++] = ent;
            }
    }
    if (B.tid == 0) { W.bptr[p] = tb; W.fptr[p] = tf; }
    __syncthreads();
}

// Levels of both solves from the dependency lists, on warp B.sw, for a
// lower-triangular selection order selrow[0..p) (Algorithms 5, 6, 8): a row's
// back-substitution step needs rows pivoting earlier columns (levels in
// selection order), its forward step needs the later rows of its pivot
// column (levels in reverse order).
template <typename T>
__device__ inline void levels_from_deps(Blk& B, WS<T>& W, int p) {
    if (B.warp == B.sw) {
        for (int k = 0; k < p; ++k) {
            const int r = W.selrow[k];
            int lv = 0;
            for (uint32_t t = W.bptr[r] + B.lane; t < W.bptr[r + 1]; t += 32)
                lv = max(lv, (int)W.lb[W.bdep[t] & kIdx]);
            lv = (int)__reduce_max_sync(kFull, (unsigned)lv) + 1;
            if (B.lane == 0) W.lb[r] = (uint16_t)lv;
            __syncwarp();
        }
        for (int k = p - 1; k >= 0; --k) {
            const int r = W.selrow[k];
            int lv = 0;
            for (uint32_t t = W.fptr[r] + B.lane; t < W.fptr[r + 1]; t += 32)
                lv = max(lv, (int)W.lf[W.fdep[t] & kIdx]);
            lv = (int)__reduce_max_sync(kFull, (unsigned)lv) + 1;
            if (B.lane == 0) W.lf[r] = (uint16_t)lv;
            __syncwarp();
        }
    }
    __syncthreads();
}

// Dependency lists, then (lower = true: from them, else already set by the
// selection) the levels of both solves, their buckets (counting sort) and
// the pivot signs. Shared by every MTS selection.
template <typename T>
__device__ inline Levels finish_levels(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                       bool lower = false) {
    const int n = C.n, p = F.p;
    build_deps<T>(B, C, W, F);
    if (lower) {
        for (int r = B.tid; r < p; r += B.nt) { W.lb[r] = 0; W.lf[r] = 0; }
        __syncthreads();
        levels_from_deps<T>(B, W, p);
    }
    int mb = 0, mf = 0;
    for (int r = B.tid; r < p; r += B.nt) {
        mb = max(mb, (int)W.lb[r]);
        mf = max(mf, (int)W.lf[r]);
        int i0 = W.pivcol[r];
        uint8_t s = 0;
        if (i0 < n) {
            for (uint32_t e = W.rptr[r]; e < W.rptr[r + 1]; ++e) {
                uint16_t ent = W.rowent[e];
                if ((ent & kIdx) == i0) s = (ent & kNeg) ? 1 : 0;
            }
        }
        W.psgn[r] = s;
    }
    mb = (int)__reduce_max_sync(kFull, (unsigned)mb);
    mf = (int)__reduce_max_sync(kFull, (unsigned)mf);
    double2 mm = bmin2(B, -(double)mb, -(double)mf);
    Levels L{(int)(-mm.x), (int)(-mm.y)};
    for (int k = B.tid; k <= max(L.nb, L.nf) + 1; k += B.nt) {
        if (k <= L.nb + 1) W.lbptr[k] = 0;
        if (k <= L.nf + 1) W.lfptr[k] = 0;
    }
    __syncthreads();
    for (int r = B.tid; r < p; r += B.nt) {
        atomicAdd(&W.lbptr[W.lb[r]], 1u);
        atomicAdd(&W.lfptr[W.lf[r]], 1u);
    }
    __syncthreads();
    if (B.tid == 0) {
        unsigned s = 0;
        for (int k = 0; k <= L.nb + 1; ++k) { unsigned c = W.lbptr[k]; W.lbptr[k] = s; s += c; }
        s = 0;
        for (int k = 0; k <= L.nf + 1; ++k) { unsigned c = W.lfptr[k]; W.lfptr[k] = s; s += c; }
    }
    __syncthreads();
    for (int k = B.tid; k <= L.nb + 1; k += B.nt) W.cur[k] = W.lbptr[k];
    __syncthreads();
    for (int r = B.tid; r < p; r += B.nt) W.lbrows[atomicAdd(&W.cur[W.lb[r]], 1u)] = (uint16_t)r;
    __syncthreads();
    for (int k = B.tid; k <= L.nf + 1; k += B.nt) W.cur[k] = W.lfptr[k];
    __syncthreads();
    for (int r = B.tid; r < p; r += B.nt) W.lfrows[atomicAdd(&W.cur[W.lf[r]], 1u)] = (uint16_t)r;
    __syncthreads();
    for (int k = B.tid; k < p; k += B.nt) {
        const int rb = W.lbrows[k], rf = W.lfrows[k];
        W.lbse[k] = make_uint2(W.bptr[rb], W.bptr[rb + 1]);
        W.lfse[k] = make_uint2(W.fptr[rf], W.fptr[rf + 1]);
    }
    __syncthreads();
    return L;
}

// Ranks the q columns by (weight desc, index asc): rank[i], sorted[k].
template <typename T>
__device__ inline void rank_columns(Blk& B, WS<T>& W, const Frame& F, const double* wt) {
    const int q = F.q;
    int q2 = 1;
    while (q2 < q) q2 <<= 1;
    // positive doubles order as their bit patterns; the complement makes the
    // ascending sort put the largest weight first (padding sorts last)
    for (int k = B.tid; k < q2; k += B.nt) {
        W.skey[k] = (k < q) ? ~(unsigned long long)__double_as_longlong(wt[k]) : ~0ull;
        W.sidx[k] = (uint32_t)k;
    }
    __syncthreads();
    bitonic_sort(B, W.skey, W.sidx, q2);
    for (int k = B.tid; k < q; k += B.nt) {
        int i = (int)W.sidx[k];
        W.rank[i] = (uint16_t)k;
        W.sorted[k] = (uint16_t)i;
    }
    __syncthreads();
}

// Back-substitution levels of an upper-triangular order, in reverse
// selection order selrow[p-1..0], on warp B.sw (every other warp returns).
template <typename T>
__device__ inline void back_levels(Blk& B, WS<T>& W, int p) {
    if (B.warp != B.sw) return;
    for (int k = p - 1; k >= 0; --k) {
        int r = W.selrow[k];
        int i0 = W.pivcol[r];
        int lv = 0;
        const int e0 = (int)W.rptr[r], d = (int)W.rptr[r + 1] - e0;
        for (int t = B.lane; t < d; t += 32) {
            int i2 = W.rowent[e0 + t] & kIdx;
            if (i2 != i0) {
                uint16_t pr = W.pivrow[i2];
                if (pr != kNone) lv = max(lv, (int)W.lb[pr]);
            }
        }
        lv = (int)__reduce_max_sync(kFull, (unsigned)lv) + 1;
        if (B.lane == 0) W.lb[r] = (uint16_t)lv;
        __syncwarp();
    }
}

template <typename T>
__device__ __noinline__ Levels mts_select(Blk& B, const CodeView C, WS<T> W, const Frame& F,
                                    const double* wt, int /*q2*/) {
    const int n = C.n, p = F.p, q = F.q;
    for (int i = B.tid; i < q; i += B.nt) {
        W.deg[i] = (uint16_t)(i < n ? (int)(W.cptr[i + 1] - W.cptr[i]) : 1);
        W.pivrow[i] = kNone;
    }
    for (int r = B.tid; r < p; r += B.nt) { W.pivcol[r] = kNone; W.lb[r] = 1; W.lf[r] = 1; }
    rank_columns<T>(B, W, F, wt);   // (barriers inside)
    const int nw = (q + 31) / 32;
    for (int k = B.tid; k < nw; k += B.nt) W.bitmap[k] = 0;
    __syncthreads();
    for (int i = B.tid; i < q; i += B.nt)
        if (W.deg[i] == 1) atomicOr(&W.bitmap[W.rank[i] >> 5], 1u << (W.rank[i] & 31));
    __syncthreads();

    if (B.warp == B.sw) {
        const int lane = B.lane;
        for (int k = 0; k < p; ++k) {
            unsigned best = 0xffffffffu;
            for (int wd = lane; wd < nw; wd += 32) {
                uint32_t v = W.bitmap[wd];
                if (v) { best = (unsigned)(wd * 32 + __ffs(v) - 1); break; }
            }
            best = __reduce_min_sync(kFull, best);
            if (best >= (unsigned)q) break;   // cannot happen: every live row keeps its slack
            int i = W.sorted[best];
            int jr, lev;
            if (i >= n) {
                jr = i - n;
                lev = 1;
            } else {
                const int beg = (int)W.cptr[i], d = (int)W.cptr[i + 1] - beg;
                unsigned cand = 0xffffffffu;
                int lv = 0;
                for (int t = lane; t < d; t += 32) {
                    int r = W.colent[beg + t] & kIdx;
                    if (W.pivcol[r] == kNone) cand = min(cand, (unsigned)r);
                    else lv = max(lv, (int)W.lf[r]);
                }
                unsigned jm = __reduce_min_sync(kFull, cand);
                lev = (int)__reduce_max_sync(kFull, (unsigned)lv) + 1;
                if (jm >= (unsigned)p) break;  // cannot happen: i has degree one
                jr = (int)jm;
            }
            __syncwarp();
            if (lane == 0) {
                W.pivcol[jr] = (uint16_t)i;
                W.pivrow[i] = (uint16_t)jr;
                W.lf[jr] = (uint16_t)lev;
                W.selrow[k] = (uint16_t)jr;
                atomicAnd(&W.bitmap[best >> 5], ~(1u << (best & 31)));
            }
            __syncwarp();
            // zero row jr: every other live column of the row loses one degree
            const int e0 = (int)W.rptr[jr], d = (int)W.rptr[jr + 1] - e0;
            for (int t = lane; t <= d; t += 32) {
                int i2 = (t < d) ? (W.rowent[e0 + t] & kIdx) : n + jr;
                if (W.pivrow[i2] != kNone) continue;   // taken (includes i)
                int nd = (int)W.deg[i2] - 1;
                W.deg[i2] = (uint16_t)nd;
                int rk = W.rank[i2];
                if (nd == 1) atomicOr(&W.bitmap[rk >> 5], 1u << (rk & 31));
                else if (nd == 0) atomicAnd(&W.bitmap[rk >> 5], ~(1u << (rk & 31)));
            }
            __syncwarp();
        }
        back_levels<T>(B, W, p);
    }
    __syncthreads();
    return finish_levels<T>(B, C, W, F);
}

// Rows of column c of the LP (its LP rows through colent; a slack column's
// only row), for warp loops: count and t-th row.
template <typename T>
__device__ __forceinline__ int col_nrows(const WS<T>& W, int n, int c) {
    return c < n ? (int)(W.cptr[c + 1] - W.cptr[c]) : 1;
}
template <typename T>
__device__ __forceinline__ int col_row(const WS<T>& W, int n, int c, int t) {
    return c < n ? (int)(W.colent[W.cptr[c] + t] & kIdx) : c - n;
}

// Lowest set bit of a bitmap of nw words, over the warp (~0u if none).
__device__ __forceinline__ unsigned warp_first_bit(const uint32_t* bm, int nw, int lane) {
    unsigned best = 0xffffffffu;
    for (int wd = lane; wd < nw; wd += 32) {
        uint32_t v = bm[wd];
        if (v) { best = (unsigned)(wd * 32 + __ffs(v) - 1); break; }
    }
    return __reduce_min_sync(kFull, best);
}

__device__ __forceinline__ void bit_set(uint32_t* bm, int i) { atomicOr(&bm[i >> 5], 1u << (i & 31)); }
__device__ __forceinline__ void bit_clear(uint32_t* bm, int i) { atomicAnd(&bm[i >> 5], ~(1u << (i & 31))); }

// ---------------------------------------------------------------------------
// a4 (variant): row-wise greedy MTS with diagonal expansion (Algorithm 8),
// on warp B.sw. While a column is left: if some row has exactly one live
// column, the lowest such row pivots it and the column is removed;
// otherwise the live column of least weight (ties: lowest index) is removed.
// Rows never pivoted then take their own slack columns in increasing order.
// The order is lower triangular. rowdeg lives in lb until the levels are
// computed.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ Levels mts_rowwise(Blk& B, const CodeView C, WS<T> W, const Frame& F,
                                     const double* wt, bool tri) {
    const int n = C.n, p = F.p, q = F.q;
    uint16_t* rowdeg = W.lb;
    for (int i = B.tid; i < q; i += B.nt) {
        W.deg[i] = (uint16_t)(col_nrows(W, n, i) > 0 ? 1 : 0);   // live
        W.pivrow[i] = kNone;
    }
    for (int r = B.tid; r < p; r += B.nt) {
        W.pivcol[r] = kNone;
        rowdeg[r] = (uint16_t)(W.rptr[r + 1] - W.rptr[r] + 1);
    }
    rank_columns<T>(B, W, F, wt);   // (barriers inside)
    const int nwr = (p + 31) / 32;
    for (int k = B.tid; k < nwr; k += B.nt) W.bitmap[k] = 0;   // rows of degree 1 (none yet)
    __syncthreads();
    if (B.warp == B.sw) {
        const int lane = B.lane;
        int live = 0;
        for (int i = lane; i < q; i += 32) live += W.deg[i];
        for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(kFull, live, o);
        int k = 0, lo = q - 1, k_round = -1;
        for (;;) {   // one search (Algorithm 8), then rounds of the triangular expansion
        while (live > 0) {
            const unsigned j = warp_first_bit(W.bitmap, nwr, lane);
            int victim;
            if (j < (unsigned)p) {
                const int e0 = (int)W.rptr[j], d = (int)W.rptr[j + 1] - e0;
                unsigned cand = 0xffffffffu;
                for (int t = lane; t <= d; t += 32) {
                    int c = (t < d) ? (W.rowent[e0 + t] & kIdx) : n + (int)j;
                    if (W.deg[c]) cand = min(cand, (unsigned)c);
                }
                const unsigned vu = __reduce_min_sync(kFull, cand);
                if (vu == 0xffffffffu) break;   // cannot happen (see above)
                victim = (int)vu;
                if (lane == 0) {
                    W.pivcol[j] = (uint16_t)victim;
                    W.pivrow[victim] = (uint16_t)j;
                    W.selrow[k] = (uint16_t)j;
                }
                ++k;
            } else {
                // least weight, then lowest index: the first live entry of
                // the run of equal weights that ends at the last live entry
                while (lo >= 0 && !W.deg[W.sorted[lo]]) --lo;
                if (lo < 0) break;              // cannot happen: a live column is left
                int t = lo;
                const double wl = wt[W.sorted[lo]];
                while (t > 0 && wt[W.sorted[t - 1]] == wl) --t;
                while (!W.deg[W.sorted[t]]) ++t;
                victim = W.sorted[t];
            }
            __syncwarp();
            if (lane == 0) W.deg[victim] = 0;
            const int nr = col_nrows(W, n, victim);
            for (int t = lane; t < nr; t += 32) {
                const int r = col_row(W, n, victim, t);
                const int nd = (int)rowdeg[r] - 1;
                rowdeg[r] = (uint16_t)nd;
                if (nd == 1) bit_set(W.bitmap, r);
                else if (nd == 0) bit_clear(W.bitmap, r);
            }
            --live;
            __syncwarp();
        }
        // triangular expansion (Section V-A): the same search again over the
        // columns with no nonzero in a row peeled so far, until every row is
        // peeled (each round peels one at least: every row left keeps its
        // slack column)
        if (!tri || k >= p || k == k_round) break;   // (a round without a peel ends it)
        k_round = k;
        int lv = 0;
        for (int c = lane; c < q; c += 32) {
            const int nr = col_nrows(W, n, c);
            int ok = nr > 0 ? 1 : 0;
            for (int t = 0; t < nr && ok; ++t)
                if (W.pivcol[col_row(W, n, c, t)] != kNone) ok = 0;
            W.deg[c] = (uint16_t)ok;
            lv += ok;
        }
        for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(kFull, lv, o);
        for (int wd = lane; wd < nwr; wd += 32) W.bitmap[wd] = 0;
        __syncwarp();
        for (int r = lane; r < p; r += 32) {
            int d = 0;
            if (W.pivcol[r] == kNone) {
                for (uint32_t e = W.rptr[r]; e < W.rptr[r + 1]; ++e) d += W.deg[W.rowent[e] & kIdx];
                d += W.deg[n + r];
            }
            rowdeg[r] = (uint16_t)d;
            if (d == 1) bit_set(W.bitmap, r);
        }
        __syncwarp();
        if (lv == 0) break;
        live = lv;
        lo = q - 1;
        }
        // diagonal expansion (rows never peeled)
        for (int base = 0; base < p; base += 32) {
            const int j = base + lane;
            const bool need = j < p && W.pivcol[j] == kNone;
            const unsigned bal = __ballot_sync(kFull, need);
            if (need) {
                const int pos = k + __popc(bal & ((1u << lane) - 1u));
                W.pivcol[j] = (uint16_t)(n + j);
                W.pivrow[n + j] = (uint16_t)j;
                W.selrow[pos] = (uint16_t)j;
            }
            k += __popc(bal);
        }
    }
    __syncthreads();
    return finish_levels<T>(B, C, W, F, true);
}

// ---------------------------------------------------------------------------
// a4 (variant): incremental greedy MTS (Algorithm 6) with the triangulation
// step (Algorithm 5), on warp B.sw. Columns are scanned by decreasing weight
// (ties: lower index) and kept when the set stays triangular, until p are
// kept. Whether S + {c} can be made lower triangular is decided exactly:
//   - if a row of c holds no column of S, c can come first (it pivots that
//     row; rows holding c only gain an earlier column): kept;
//   - if no row of c is the pivot row of a column of S (under the current
//     assignment of pivot rows), c can come last, pivoting its lowest row:
//     kept;
//   - otherwise by peeling S + {c} (Algorithm 5: a row with exactly one live
//     column pivots it; the set is triangular iff every column peels), whose
//     pivots become the new assignment when it succeeds.
// The final (column, row) pairs and order are those of Algorithm 5 on the
// kept set with the lowest-index degree-1 row taken at each step. Scratch:
// rowcnt (S columns per row) in lb, live-row counts in lf, live stamps in
// rank, the set S in lbrows, the peel's rows / columns in lfrows / cchk2, a
// stack of degree-1 rows in selrow.
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline int peel_set(Blk& B, WS<T>& W, int n, int p, int s, uint16_t stamp,
                               bool lowest_first) {
    // live columns (S, stamped) of every row; degree-1 rows on a stack (or,
    // for the lowest-first order, in the bitmap)
    const int lane = B.lane;
    uint16_t* cnt = W.lf;
    uint16_t* stk = W.selrow;
    int top = 0;
    const int nwr = (p + 31) / 32;
    if (lowest_first)
        for (int k = lane; k < nwr; k += 32) W.bitmap[k] = 0;
    __syncwarp();
    for (int base = 0; base < p; base += 32) {
        const int r = base + lane;
        int c = 0;
        if (r < p) {
            for (uint32_t e = W.rptr[r]; e < W.rptr[r + 1]; ++e)
                c += W.rank[W.rowent[e] & kIdx] == stamp;
            c += W.rank[n + r] == stamp;
            cnt[r] = (uint16_t)c;
        }
        const unsigned bal = __ballot_sync(kFull, r < p && c == 1);
        if (r < p && c == 1) {
            if (lowest_first) bit_set(W.bitmap, r);
            else stk[top + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)r;
        }
        top += __popc(bal);
    }
    __syncwarp();
    int peeled = 0;
    for (;;) {
        int j;
        if (lowest_first) {
            const unsigned b = warp_first_bit(W.bitmap, nwr, lane);
            if (b >= (unsigned)p) break;
            j = (int)b;
        } else {
            if (top == 0) break;
            j = stk[--top];
            if (cnt[j] != 1) continue;   // (uniform: every lane reads the same)
        }
        const int e0 = (int)W.rptr[j], d = (int)W.rptr[j + 1] - e0;
        unsigned cand = 0xffffffffu;
        for (int t = lane; t <= d; t += 32) {
            int c = (t < d) ? (W.rowent[e0 + t] & kIdx) : n + j;
            if (W.rank[c] == stamp) cand = min(cand, (unsigned)c);
        }
        const unsigned xu = __reduce_min_sync(kFull, cand);
        if (xu == 0xffffffffu) break;   // cannot happen: a degree-1 row holds one live column
        const int x = (int)xu;
        __syncwarp();
        if (lane == 0) {
            W.rank[x] = 0;
            W.lfrows[peeled] = (uint16_t)j;
            W.cchk2[peeled] = (uint16_t)x;
        }
        ++peeled;
        const int nr = col_nrows(W, n, x);
        for (int base = 0; base < nr; base += 32) {   // uniform trip count
            const int t = base + lane;
            int pr = -1;
            if (t < nr) {
                const int r = col_row(W, n, x, t);
                const int nd = (int)cnt[r] - 1;
                cnt[r] = (uint16_t)nd;
                if (lowest_first) {
                    if (nd == 1) bit_set(W.bitmap, r);
                    else if (nd == 0) bit_clear(W.bitmap, r);
                } else if (nd == 1) {
                    pr = r;
                }
            }
            if (!lowest_first) {
                const unsigned bal = __ballot_sync(kFull, pr >= 0);
                if (pr >= 0) stk[top + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)pr;
                top += __popc(bal);
            }
        }
        __syncwarp();
    }
    (void)s;
    return peeled;
}

template <typename T>
__device__ __noinline__ Levels mts_incremental(Blk& B, const CodeView C, WS<T> W, const Frame& F,
                                         const double* wt) {
    const int n = C.n, p = F.p, q = F.q;
    uint16_t* rowcnt = W.lb;
    for (int i = B.tid; i < q; i += B.nt) { W.pivrow[i] = kNone; W.deg[i] = 0; }
    for (int r = B.tid; r < p; r += B.nt) { W.pivcol[r] = kNone; rowcnt[r] = 0; }
    rank_columns<T>(B, W, F, wt);   // (barriers inside)
    for (int i = B.tid; i < q; i += B.nt) W.rank[i] = 0;   // live stamps from here on
    __syncthreads();
    if (B.warp == B.sw) {
        const int lane = B.lane;
        int s = 0;
        uint16_t stamp = 0;
        for (int k = 0; k < q && s < p; ++k) {
            const int c = W.sorted[k];
            const int nr = col_nrows(W, n, c);
            if (nr == 0) continue;                 // a zero column is never triangular
            unsigned empty = 0xffffffffu, any = 0xffffffffu;
            int piv = 0;
            for (int t = lane; t < nr; t += 32) {
                const int r = col_row(W, n, c, t);
                if (rowcnt[r] == 0) empty = min(empty, (unsigned)r);
                any = min(any, (unsigned)r);
                piv |= W.pivcol[r] != kNone;
            }
            empty = __reduce_min_sync(kFull, empty);
            any = __reduce_min_sync(kFull, any);
            piv = __any_sync(kFull, piv);
            bool keep = false;
            if (empty < (unsigned)p || !piv) {
                const int r0 = (int)(empty < (unsigned)p ? empty : any);
                __syncwarp();
                if (lane == 0) { W.pivcol[r0] = (uint16_t)c; W.pivrow[c] = (uint16_t)r0; }
                keep = true;
            } else {
                // Algorithm 5 on S + {c}
                if (++stamp == 0) {            // (never with q < 65535 candidates)
                    for (int i = lane; i < q; i += 32) W.rank[i] = 0;
                    stamp = 1;
                }
                __syncwarp();
                for (int t = lane; t < s; t += 32) W.rank[W.lbrows[t]] = stamp;
                if (lane == 0) W.rank[c] = stamp;
                __syncwarp();
                const int peeled = peel_set<T>(B, W, n, p, s + 1, stamp, false);
                if (peeled == s + 1) {
                    for (int r = lane; r < p; r += 32) W.pivcol[r] = kNone;
                    __syncwarp();
                    for (int t = lane; t < peeled; t += 32) {
                        const int j = W.lfrows[t], x = W.cchk2[t];
                        W.pivcol[j] = (uint16_t)x;
                        W.pivrow[x] = (uint16_t)j;
                    }
                    keep = true;
                }
            }
            if (keep) {
                for (int t = lane; t < nr; t += 32) {
                    const int r = col_row(W, n, c, t);
                    rowcnt[r] = (uint16_t)(rowcnt[r] + 1);
                }
                if (lane == 0) { W.lbrows[s] = (uint16_t)c; W.deg[c] = 1; }
                ++s;
            }
            __syncwarp();
        }
        // final pairs and order: Algorithm 5 on the kept set, lowest-index
        // degree-1 row first
        if (++stamp == 0) {
            for (int i = lane; i < q; i += 32) W.rank[i] = 0;
            stamp = 1;
        }
        __syncwarp();
        for (int t = lane; t < s; t += 32) W.rank[W.lbrows[t]] = stamp;
        for (int r = lane; r < p; r += 32) W.pivcol[r] = kNone;
        __syncwarp();
        const int peeled = peel_set<T>(B, W, n, p, s, stamp, true);
        for (int t = lane; t < peeled; t += 32) {
            const int j = W.lfrows[t], x = W.cchk2[t];
            W.pivcol[j] = (uint16_t)x;
            W.pivrow[x] = (uint16_t)j;
            W.selrow[t] = (uint16_t)j;
        }
        __syncwarp();
        // (defensive: Algorithm 6 always keeps p columns; a row left without
        // a pivot would take its own slack column, which keeps the set
        // triangular)
        int k = peeled;
        for (int base = 0; base < p; base += 32) {
            const int j = base + lane;
            const bool need = j < p && W.pivcol[j] == kNone;
            const unsigned bal = __ballot_sync(kFull, need);
            if (need) {
                W.pivcol[j] = (uint16_t)(n + j);
                W.pivrow[n + j] = (uint16_t)j;
                W.selrow[k + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)j;
            }
            k += __popc(bal);
        }
    }
    __syncthreads();
    return finish_levels<T>(B, C, W, F, true);
}

// The preconditioner of one Newton system: Algorithm 7 (column-wise), 6
// (incremental) or 8 (row-wise).
template <typename T>
__device__ inline Levels select_mts(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                    const double* wt, int kind) {
    if (kind == LPDEC_MTS_INCREMENTAL) return mts_incremental<T>(B, C, W, F, wt);
    if (kind == LPDEC_MTS_ROWWISE || kind == LPDEC_MTS_ROWWISE_TRI)
        return mts_rowwise<T>(B, C, W, F, wt, kind == LPDEC_MTS_ROWWISE_TRI);
    return mts_select<T>(B, C, W, F, wt, 0);
}

// Selection order as (column, row) pairs, for the step entry point.
template <typename T>
__device__ inline void selection_order(Blk& B, WS<T>& W, const Frame& F, int32_t* col,
                                       int32_t* row, int m) {
    for (int k = B.tid; k < m; k += B.nt) {
        int r = k < F.p ? (int)W.selrow[k] : -1;
        row[k] = r;
        col[k] = r >= 0 ? (int)W.pivcol[r] : -1;
    }
}

// One row of a triangular solve, reduced by a group of G lanes (G a power
// of two <= 32, g = lane index inside the group): the group sums its share
// of the row's dependencies and the leader (g == 0) finishes the row. Back:
// out[r] = +-(r_r - sum); forward: out[r] = +-(out[r] / d_piv - sum). All 32
// lanes of the warp call this (r < 0 marks an idle group).
// One row of a triangular solve, reduced by a group of G lanes (G a power
// of two <= 32, g = lane index inside the group). The lane sums its share of
// the row's dependencies (entries begin + g, begin + g + G, ...; the first
// two, d0 and d1, already loaded, kNone when absent) and the group reduces;
// the leader (g == 0) finishes the row. Back: out[r] = +-(r_r - sum);
// forward: out[r] = +-(out[r] / d_piv - sum). All 32 lanes of the warp call
// this (r < 0 marks an idle group).
template <typename T, bool kBack, bool kScale = true>
__device__ __forceinline__ void solve_row(WS<T>& W, const uint16_t* dep, int r, uint32_t e,
                                          uint32_t k2, uint16_t d0, uint16_t d1, int G, int g,
                                          T* rvec, T* out, T alpha) {
    T acc = T(0);
    if (d0 != kNone) acc += signed_val<T>(d0, out[d0 & kIdx]);
    if (d1 != kNone) acc += signed_val<T>(d1, out[d1 & kIdx]);
    for (uint32_t k = k2; k < e; k += G) {
        const uint16_t ent = dep[k];
        acc += signed_val<T>(ent, out[ent & kIdx]);
    }
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o, G);
    if (r >= 0 && g == 0) {
        T v;
        if (kBack) {
            T rv = rvec[r];
            if (alpha != T(0)) {
                rv -= alpha * W.l[r];
                rvec[r] = rv;
                W.xs[r] += alpha * W.h[r];
            }
            v = rv - acc;
        } else {
            v = (kScale ? out[r] * W.invd2p[r] : out[r]) - acc;
        }
        out[r] = W.psgn[r] ? -v : v;
    }
}

// The row at level position idx (< end) for lane group g of size G: its
// index, dependency range and first two dependency entries of the lane.
struct RowSlot {
    int r;
    uint32_t e, k2;
    uint16_t d0, d1;
};
__device__ __forceinline__ RowSlot load_slot(const uint16_t* rows, const uint2* se,
                                             const uint16_t* dep, int idx, int end, int G, int g) {
    RowSlot t{-1, 0u, 0u, kNone, kNone};
    if (idx < end) {
        t.r = rows[idx];
        const uint2 v = se[idx];
        const uint32_t k0 = v.x + g;
        t.e = v.y;
        t.d0 = k0 < v.y ? dep[k0] : kNone;
        t.d1 = k0 + G < v.y ? dep[k0 + G] : kNone;
        t.k2 = k0 + 2 * G;
    }
    return t;
}

// Lanes per row of a warp-mode level of cnt rows: by the level's width
// (policy 0: 8 lanes for up to 4 rows, 4 up to 8, 2 up to 16, else 1) or a
// fixed 1, 2, 4 or 8 (the schedule the autotuner picks, lpdec_autotune).
__device__ __forceinline__ int group_of(int cnt, int policy) {
    if (policy == 1 || policy == 2 || policy == 4 || policy == 8) return policy;
    return cnt <= 4 ? 8 : cnt <= 8 ? 4 : cnt <= 16 ? 2 : 1;
}

// Runs rows level by level. Levels wider than two warps use every thread of
// the CTA (one row per thread) and a CTA barrier; narrower levels (most of
// them: the schedules are deep and thin) run on one warp (B.sw) with G lanes
// per row and warp barriers. On that warp the next level's first rows (row,
// dependency range, the lane's first two dependency entries: none of them
// depends on the values being solved) are loaded before the current level's
// barrier, so a level's dependent chain starts at the solved values.
template <typename T, bool kBack, bool kScale = true>
__device__ inline void level_sweep(Blk& B, WS<T>& W, const uint32_t* ptr, const uint16_t* rows,
                                   const uint2* se, int nlev, T* rvec, T* out, T alpha) {
    const uint16_t* dep = kBack ? W.bdep : W.fdep;
    bool warp_mode = false;
    RowSlot pre{-1, 0u, 0u, kNone, kNone};
    bool have_pre = false;   // pre holds the first pass of the level about to run
    int i1 = nlev >= 1 ? (int)ptr[1] : 0;
    for (int lev = 1; lev <= nlev; ++lev) {
        const int i0 = i1;
        i1 = ptr[lev + 1];
        const int cnt = i1 - i0;
        if (cnt > 64 && B.nt > 32) {
            if (warp_mode) __syncthreads();
            for (int base = i0; base < i1; base += B.nt) {   // uniform trip count per warp
                const RowSlot t = load_slot(rows, se, dep, base + B.tid, i1, 1, 0);
                solve_row<T, kBack, kScale>(W, dep, t.r, t.e, t.k2, t.d0, t.d1, 1, 0, rvec, out,
                                            alpha);
            }
            __syncthreads();
            warp_mode = false;
            have_pre = false;
        } else {
            if (B.warp == B.sw) {
                const int G = group_of(cnt, W.lanes);
                const int per = 32 / G, g = B.lane & (G - 1);
                for (int base = i0; base < i1; base += per) {
                    const RowSlot t = (base == i0 && have_pre)
                                          ? pre
                                          : load_slot(rows, se, dep, base + B.lane / G, i1, G, g);
                    solve_row<T, kBack, kScale>(W, dep, t.r, t.e, t.k2, t.d0, t.d1, G, g, rvec,
                                                out, alpha);
                }
                // next level's first pass, if it runs on this warp
                have_pre = false;
                if (lev < nlev) {
                    const int n1 = ptr[lev + 2], c1 = n1 - i1;
                    if (!(c1 > 64 && B.nt > 32)) {
                        const int G1 = group_of(c1, W.lanes);
                        pre = load_slot(rows, se, dep, i1 + B.lane / G1, n1, G1, B.lane & (G1 - 1));
                        have_pre = true;
                    }
                }
                __syncwarp();
            }
            warp_mode = true;
        }
    }
    if (warp_mode) __syncthreads();
}

// The same two sweeps in FP32 on the M-solve vectors rf -> zf (LPDEC_M32):
// no fused PCG update, so the serial chain of each level holds only FP32
// arithmetic (GB300's FP64 pipe retires a warp instruction every few dozen
// cycles, FP32 every cycle).
template <bool kBack, typename T>
__device__ __forceinline__ void solve_row32(WS<T>& W, int r, int g, int G) {
    float acc = 0.0f;
    if (r >= 0) {
        const uint32_t* ptr = kBack ? W.bptr : W.fptr;
        const uint16_t* dep = kBack ? W.bdep : W.fdep;
        const int k1 = ptr[r + 1];
        for (int k = ptr[r] + g; k < k1; k += G) {
            uint16_t ent = dep[k];
            float v = W.zf[ent & kIdx];
            acc += (ent & kNeg) ? -v : v;
        }
    }
    for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o, G);
    if (r >= 0 && g == 0) {
        float v = (kBack ? W.rf[r] : W.zf[r] * W.ip32[r]) - acc;
        W.zf[r] = W.psgn[r] ? -v : v;
    }
}

template <bool kBack, typename T>
__device__ inline void level_sweep32(Blk& B, WS<T>& W, const uint32_t* ptr, const uint16_t* rows,
                                     int nlev) {
    bool warp_mode = false;
    for (int lev = 1; lev <= nlev; ++lev) {
        const int i0 = ptr[lev], i1 = ptr[lev + 1];
        const int cnt = i1 - i0;
        if (cnt > 64 && B.nt > 32) {
            if (warp_mode) __syncthreads();
            for (int base = i0; base < i1; base += B.nt) {
                int idx = base + B.tid;
                solve_row32<kBack>(W, idx < i1 ? rows[idx] : -1, 0, 1);
            }
            __syncthreads();
            warp_mode = false;
        } else {
            if (B.warp == B.sw) {
                const int G = cnt <= 4 ? 8 : cnt <= 8 ? 4 : cnt <= 16 ? 2 : 1;
                const int per = 32 / G;
                for (int base = i0; base < i1; base += per) {
                    int idx = base + B.lane / G;
                    solve_row32<kBack>(W, idx < i1 ? rows[idx] : -1, B.lane & (G - 1), G);
                }
                __syncwarp();
            }
            warp_mode = true;
        }
    }
    if (warp_mode) __syncthreads();
}

// ---------------------------------------------------------------------------
// a5: M-solve (Section V): A_M f1 = r by back substitution over the upper-
// triangular order of Algorithm 7, f2 = f1 / d_M^2, then A_M' z = f2 by
// forward substitution. out[r] first holds the value of r's pivot column in
// f1, then z_r. If alpha != 0, the PCG update r -= alpha l, xs += alpha h of
// each row is fused into its back-substitution step.
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline void msolve(Blk& B, const CodeView& C, WS<T>& W, const Levels& L,
                              T* rvec, T* out, T alpha) {
    level_sweep<T, true>(B, W, W.lbptr, W.lbrows, W.lbse, L.nb, rvec, out, alpha);
    level_sweep<T, false>(B, W, W.lfptr, W.lfrows, W.lfse, L.nf, rvec, out, alpha);
}

// M-solve in FP32: zf = M^-1 rf (rf written by the caller before a barrier).
template <typename T>
__device__ inline void msolve32(Blk& B, WS<T>& W, const Levels& L) {
    level_sweep32<true>(B, W, W.lbptr, W.lbrows, L.nb);
    level_sweep32<false>(B, W, W.lfptr, W.lfrows, L.nf);
}

// l = Q h = A D^2 A' h (matrix-free; t holds D^2 A' h over the standard
// columns). Returns h'l in FP64.
template <typename T>
__device__ inline double spmv_Q(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                const T* hv, T* lv) {
    const int n = C.n;
    for (int i = B.tid; i < n; i += B.nt) W.t[i] = W.d2t[i] * colA_T<T>(C, W, i, hv);
    __syncthreads();
    double hl = 0.0;
    for (int r = B.tid; r < F.p; r += B.nt) {
        T v = rowA<T>(C, W, r, W.t) + W.d2t[n + r] * hv[r];
        lv[r] = v;
        hl += (double)hv[r] * (double)v;
    }
    return bsum(B, hl);
}

// Record of CG coefficients for the Lanczos estimate of a traced solve:
// lz[2k] = alpha_k, lz[2k+1] = nu_k (k < kLz), lz[2 kLz] = count,
// lz[2 kLz + 1] = 1 once the first PCG round has ended.
constexpr int kLz = 64;
__device__ __forceinline__ void lz_record(double* lz, double alpha, double nu) {
    const int k = (int)lz[2 * kLz];
    if (lz[2 * kLz + 1] == 0.0 && k < kLz) {
        lz[2 * k] = alpha;
        lz[2 * k + 1] = nu;
        lz[2 * kLz] = k + 1;
    }
}

// Extreme eigenvalues of the Lanczos tridiagonal of the recorded CG
// coefficients (diagonal 1/alpha_k + nu_{k-1}/alpha_{k-1}, off-diagonal
// sqrt(nu_k)/alpha_k), by bisection on Sturm counts inside the Gershgorin
// interval (one thread).
__device__ inline void lz_extremes(const double* lz, double* lo, double* hi) {
    const int k = (int)lz[2 * kLz];
    *lo = *hi = NAN;
    if (k < 1) return;
    double d[kLz], e[kLz];
    double gl = INFINITY, gh = -INFINITY;
    for (int j = 0; j < k; ++j) {
        d[j] = 1.0 / lz[2 * j] + (j > 0 ? lz[2 * j - 1] / lz[2 * j - 2] : 0.0);
        e[j] = j + 1 < k ? sqrt(fmax(lz[2 * j + 1], 0.0)) / lz[2 * j] : 0.0;
    }
    for (int j = 0; j < k; ++j) {
        const double rad = fabs(e[j]) + (j > 0 ? fabs(e[j - 1]) : 0.0);
        gl = fmin(gl, d[j] - rad);
        gh = fmax(gh, d[j] + rad);
    }
    auto below = [&](double x) {   // eigenvalues < x
        int c = 0;
        double q = d[0] - x;
        if (q < 0.0) ++c;
        for (int j = 1; j < k; ++j) {
            const double qq = (q == 0.0) ? 1e-300 : q;
            q = d[j] - x - e[j - 1] * e[j - 1] / qq;
            if (q < 0.0) ++c;
        }
        return c;
    };
    for (int which = 0; which < 2; ++which) {   // 0: smallest, 1: largest
        double a = gl, b = gh;
        for (int t = 0; t < 200 && b - a > 1e-14 * fmax(fabs(a), fabs(b)); ++t) {
            const double mid = 0.5 * (a + b);
            const bool left = which == 0 ? below(mid) >= 1 : below(mid) >= k;
            if (left) b = mid; else a = mid;
        }
        if (which == 0) *lo = 0.5 * (a + b); else *hi = 0.5 * (a + b);
    }
}

// PCG (Algorithm 4) in type T on Q xs = r (right side in W.r, overwritten by
// the residual), x0 = 0, stopping when ||r||_2 < tol ||rhs||_2 or after
// max_it iterations. Dot products accumulate in FP64.
template <typename T>
__device__ inline int pcg_m32(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                              const Levels& L, double tol, int max_it, double* relres);

template <typename T>
__device__ inline int pcg(Blk& B, const CodeView& C, WS<T>& W, const Frame& F, const Levels& L,
                          double tol, int max_it, double* relres, bool m32 = false) {
    if (m32) return pcg_m32<T>(B, C, W, F, L, tol, max_it, relres);
    const int p = F.p;
    for (int r = B.tid; r < p; r += B.nt) W.xs[r] = T(0);
    __syncthreads();
    msolve<T>(B, C, W, L, W.r, W.z, T(0));
    double zr0 = 0.0, rr0 = 0.0;
    for (int r = B.tid; r < p; r += B.nt) {
        W.h[r] = W.z[r];
        zr0 += (double)W.z[r] * (double)W.r[r];
        rr0 += (double)W.r[r] * (double)W.r[r];
    }
    double2 s = bsum2(B, zr0, rr0);
    double zr = s.x, rr = s.y;
    const double rn0 = sqrt(rr);
    *relres = 0.0;
    if (rn0 == 0.0) return 0;
    int it = 0;
    while (sqrt(rr) >= tol * rn0 && it < max_it) {
        double hl = spmv_Q<T>(B, C, W, F, W.h, W.l);
        if (!(hl > 0.0) || !isfinite(hl)) break;   // lost positive curvature (rounding)
        T alpha = (T)(zr / hl);
        // r -= a l, xs += a h over all warps, then the M-solve: the serial
        // sweeps keep only the substitution itself
        for (int r = B.tid; r < p; r += B.nt) {
            W.r[r] -= alpha * W.l[r];
            W.xs[r] += alpha * W.h[r];
        }
        __syncthreads();
        msolve<T>(B, C, W, L, W.r, W.z, T(0));
        double zr_l = 0.0, rr_l = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            zr_l += (double)W.z[r] * (double)W.r[r];
            rr_l += (double)W.r[r] * (double)W.r[r];
        }
        s = bsum2(B, zr_l, rr_l);
        T nu = (T)(s.x / zr);
        if (W.lz && B.tid == 0) lz_record(W.lz, (double)alpha, s.x / zr);
        zr = s.x;
        rr = s.y;
        for (int r = B.tid; r < p; r += B.nt) W.h[r] = W.z[r] + nu * W.h[r];
        __syncthreads();
        ++it;
    }
    if (W.lz && B.tid == 0) W.lz[2 * kLz + 1] = 1.0;   // later rounds are not recorded
    *relres = isfinite(rr) ? sqrt(rr) / rn0 : INFINITY;
    return it;
}

// Diagnostic PCG (Algorithm 4) in FP64 on Q xs = r (right side in W.r),
// x0 = 0, that records per iteration k < max_hist: hist[3k] = ||r_k|| /
// ||r_0||, hist[3k+1] = alpha_k, hist[3k+2] = nu_k. The coefficients give the
// Lanczos tridiagonal of the preconditioned operator M^-1 Q, whose extreme
// eigenvalues estimate its condition number. identity = true runs plain CG
// (M = I). Stops at ||r|| < tol ||r_0|| or after max_hist iterations.
template <typename T>
__device__ inline int pcg_traced(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                 const Levels& L, bool identity, double tol, int max_hist,
                                 double* hist) {
    const int p = F.p;
    auto apply_m = [&]() {
        if (identity) {
            for (int r = B.tid; r < p; r += B.nt) W.z[r] = W.r[r];
            __syncthreads();
        } else {
            msolve<T>(B, C, W, L, W.r, W.z, T(0));
        }
    };
    for (int r = B.tid; r < p; r += B.nt) W.xs[r] = T(0);
    __syncthreads();
    apply_m();
    double zr0 = 0.0, rr0 = 0.0;
    for (int r = B.tid; r < p; r += B.nt) {
        W.h[r] = W.z[r];
        zr0 += (double)W.z[r] * (double)W.r[r];
        rr0 += (double)W.r[r] * (double)W.r[r];
    }
    double2 s = bsum2(B, zr0, rr0);
    double zr = s.x, rr = s.y;
    const double rn0 = sqrt(rr);
    if (rn0 == 0.0) return 0;
    int it = 0;
    while (sqrt(rr) >= tol * rn0 && it < max_hist) {
        double hl = spmv_Q<T>(B, C, W, F, W.h, W.l);
        if (!(hl > 0.0) || !isfinite(hl)) break;
        const double alpha = zr / hl;
        for (int r = B.tid; r < p; r += B.nt) {
            W.r[r] -= (T)alpha * W.l[r];
            W.xs[r] += (T)alpha * W.h[r];
        }
        __syncthreads();
        apply_m();
        double zr_l = 0.0, rr_l = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            zr_l += (double)W.z[r] * (double)W.r[r];
            rr_l += (double)W.r[r] * (double)W.r[r];
        }
        s = bsum2(B, zr_l, rr_l);
        const double nu = s.x / zr;
        zr = s.x;
        rr = s.y;
        for (int r = B.tid; r < p; r += B.nt) W.h[r] = W.z[r] + (T)nu * W.h[r];
        if (B.tid == 0) {
            hist[3 * it] = sqrt(rr) / rn0;
            hist[3 * it + 1] = alpha;
            hist[3 * it + 2] = nu;
        }
        __syncthreads();
        ++it;
    }
    return it;
}

__device__ inline double3 bsum3(Blk& B, double a, double b, double c) {
    double2 ab = bsum2(B, a, b);
    return make_double3(ab.x, ab.y, bsum(B, c));
}

// PCG of LPDEC_M32: the Krylov recurrences, Q h and the dot products in
// FP64 (type T = double), the preconditioner M^-1 (the two triangular
// sweeps) in FP32. An FP32 M-solve is a slightly perturbed, not exactly
// symmetric preconditioner, so the direction update uses the flexible
// (Polak-Ribiere) coefficient nu = z_{k+1}'(r_{k+1} - r_k) / z_k'r_k
// = -alpha z_{k+1}'l_k / z_k'r_k, which equals the Fletcher-Reeves value
// of Algorithm 4 when M^-1 is applied exactly.
template <typename T>
__device__ inline int pcg_m32(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                              const Levels& L, double tol, int max_it, double* relres) {
    const int p = F.p;
    for (int r = B.tid; r < p; r += B.nt) { W.xs[r] = T(0); W.rf[r] = (float)W.r[r]; }
    __syncthreads();
    msolve32<T>(B, W, L);
    double zr0 = 0.0, rr0 = 0.0;
    for (int r = B.tid; r < p; r += B.nt) {
        const double zv = (double)W.zf[r];
        W.h[r] = (T)zv;
        zr0 += zv * (double)W.r[r];
        rr0 += (double)W.r[r] * (double)W.r[r];
    }
    double2 s = bsum2(B, zr0, rr0);
    double zr = s.x, rr = s.y;
    const double rn0 = sqrt(rr);
    *relres = 0.0;
    if (rn0 == 0.0) return 0;
    int it = 0;
    while (sqrt(rr) >= tol * rn0 && it < max_it) {
        double hl = spmv_Q<T>(B, C, W, F, W.h, W.l);
        if (!(hl > 0.0) || !isfinite(hl) || !(zr > 0.0)) break;
        const double alpha = zr / hl;
        for (int r = B.tid; r < p; r += B.nt) {
            const double rv = (double)W.r[r] - alpha * (double)W.l[r];
            W.r[r] = (T)rv;
            W.xs[r] = (T)((double)W.xs[r] + alpha * (double)W.h[r]);
            W.rf[r] = (float)rv;
        }
        __syncthreads();
        msolve32<T>(B, W, L);
        double zr_l = 0.0, rr_l = 0.0, zl_l = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            const double zv = (double)W.zf[r];
            zr_l += zv * (double)W.r[r];
            rr_l += (double)W.r[r] * (double)W.r[r];
            zl_l += zv * (double)W.l[r];
        }
        double3 s3 = bsum3(B, zr_l, rr_l, zl_l);
        const double nu = -alpha * s3.z / zr;
        zr = s3.x;
        rr = s3.y;
        for (int r = B.tid; r < p; r += B.nt) W.h[r] = (T)((double)W.zf[r] + nu * (double)W.h[r]);
        __syncthreads();
        ++it;
    }
    *relres = isfinite(rr) ? sqrt(rr) / rn0 : INFINITY;
    return it;
}

// Newton solve (A D^2 A') dy = w with iterative refinement: each round
// solves Q d = r64 / ||r64|| by PCG, adds ||r64|| d to the FP64 solution dy
// and recomputes the FP64 residual r64 = w - Q dy with FP64 D^2. Rounds run
// in type T; in the mixed mode (T = float), once an FP32 round fails to
// reach its tolerance or to halve ||r64||, the remaining rounds run in FP64
// (FP32 cannot resolve the preconditioned system once D^2 spreads over many
// decades near the optimum). Stops at ||r64|| < tol ||w||, when an FP64
// round no longer halves ||r64||, or when the PCG budget is spent.
struct NewtonOut { int iters, iters64, dense; double relres, flops, bytes; };

// Algorithmic floating-point operations of one PCG iteration (Algorithm 4):
// Q h (2 passes over the pattern, D^2 and the slacks), the two triangular
// solves (one multiply-add per dependency, pivot scaling), three dot
// products and the vector updates.
// Algorithmic bytes of one PCG iteration, as the survey's roofline counts
// them for a streamed frame (4-byte indices, FP64 D^2, vectors of rb bytes):
// Q h reads both index passes (8 E_A), the row list (4p), D^2 (8q) and h,
// and writes l; each triangular solve reads 4 nnz(A_M) + 8p; two dot
// products and three vector updates move 5 vectors of 8p.
__device__ __forceinline__ double pcg_iter_bytes(const Frame& F, int n, int nnz_m, int rb) {
    const double p = F.p;
    return 8.0 * F.ea + 4.0 * p + 8.0 * (n + p) + 2.0 * rb * p + 2.0 * (4.0 * nnz_m + 8.0 * p) +
           40.0 * p;
}
__device__ __forceinline__ double pcg_iter_flops(const Frame& F, int n, int deps) {
    return 4.0 * F.ea + 2.0 * deps + n + 15.0 * F.p;
}
// ... and of one dense fallback solve: forming Q, the Cholesky
// factorization (p^3 / 3), two triangular solves and the FP64 residual.
__device__ __forceinline__ double dense_flops(const Frame& F, int n) {
    const double p = F.p;
    return p * p * p / 3.0 + 2.0 * p * p + 4.0 * F.ea + n + 3.0 * p;
}

template <typename V, typename T>
__device__ inline void residual64(Blk& B, const CodeView& C, WS<T>& W, const Frame& F, double* rr) {
    const int n = C.n, p = F.p;
    for (int i = B.tid; i < n; i += B.nt) W.t64[i] = W.d2[i] * colA_T<double>(C, W, i, W.dy);
    __syncthreads();
    double acc = 0.0;
    for (int r = B.tid; r < p; r += B.nt) {
        double v = W.w[r] - (rowA<double>(C, W, r, W.t64) + W.d2[n + r] * W.dy[r]);
        W.r64[r] = v;
        acc += v * v;
    }
    *rr = bsum(B, acc);
}

template <typename V, typename T>
__device__ inline int refine_round(Blk& B, const CodeView& C, WS<V>& WV, WS<T>& W, const Frame& F,
                                   const Levels& L, double rn, double target, int budget,
                                   double* rel, bool m32 = false) {
    const int p = F.p;
    const double inv = 1.0 / rn;
    for (int r = B.tid; r < p; r += B.nt) WV.r[r] = (V)(W.r64[r] * inv);
    __syncthreads();
    int it = pcg<V>(B, C, WV, F, L, target, budget, rel, m32);
    int bad = 0;
    for (int r = B.tid; r < p; r += B.nt) bad |= !isfinite((double)WV.xs[r]);
    bad = __syncthreads_or(bad);
    if (bad) {            // overflow in this precision: keep dy, report failure
        *rel = INFINITY;
        return it;
    }
    for (int r = B.tid; r < p; r += B.nt) W.dy[r] += rn * (double)WV.xs[r];
    __syncthreads();
    return it;
}

// Fallback Newton solve (A D^2 A') dy = w by a dense FP64 Cholesky
// factorization Q = L L' (column-major, leading dimension p, in W.qd), for
// the systems on which PCG stalls or runs long (large degenerate LPs near
// the optimum, where the MTS preconditioner of Section V no longer captures
// Q). This is the direct method of the normal equations (Eq. 24); it leaves
// dy untouched and returns false if Q has a non-finite entry or a
// non-positive diagonal.
//
// Blocked right-looking factorization, panels of kDB = 32 columns: the
// panel's diagonal block is factored by one warp; the rows below it are
// solved against that block, one row per thread (32 values in registers);
// the trailing lower triangle is updated in 4 x 4 register tiles, one tile
// per thread at a time, reading the panel from L2 (consecutive threads take
// consecutive row tiles of one column tile, so the loads coalesce). The two
// triangular solves go panel by panel as well: one warp solves the 32 x 32
// diagonal block, then every thread updates its rows. Each panel costs a
// few CTA barriers instead of one or two per column.
constexpr double kPivotTiny = 1e-13;
constexpr double kPivotHuge = 1e64;
constexpr int kDB = 32;

// Factors columns k0 .. k0+kb-1 of the diagonal block in place (one warp;
// lane l holds row k0+j+1+l of column j). The original diagonal of column
// j >= 1 is kept at (j-1, j), in the unused upper triangle. Returns true
// (same in every lane) if a diagonal entry is non-finite or not positive.
__device__ __forceinline__ bool chol_diag_block(double* A, int p, int k0, int kb, int lane) {
    bool bad = false;
    for (int j = 0; j < kb; ++j) {
        const int jj = k0 + j;
        double* colj = A + (size_t)jj * p;
        const double sjj = colj[jj];
        const double qjj = jj == 0 ? sjj : colj[jj - 1];
        bad = bad || !isfinite(sjj) || !(qjj > 0.0);
        // A pivot at the rounding level of Q(j,j) means Q is singular to
        // working precision along y_j (a degenerate optimum): it is given a
        // huge value, which zeroes that component of the step instead of
        // amplifying rounding noise (the usual treatment of tiny pivots in
        // interior-point normal equations).
        const bool tiny = !(sjj > kPivotTiny * qjj);
        const double ljj = tiny ? kPivotHuge : sqrt(sjj), inv = 1.0 / ljj;
        const int i = jj + 1 + lane;
        double lij = 0.0;
        if (i < k0 + kb) { lij = colj[i] * inv; colj[i] = lij; }
        __syncwarp();
        if (lane == 0) colj[jj] = ljj;
        if (i < k0 + kb)
            for (int l = jj + 1; l <= i; ++l) A[(size_t)l * p + i] -= lij * colj[l];
        __syncwarp();
    }
    return bad;
}

template <typename T>
__device__ __noinline__ bool dense_newton(Blk& B, const CodeView C, WS<T> W, const Frame& F) {
    const int n = C.n, p = F.p;
    double* A = W.qd;
    const size_t pp = (size_t)p * p;
    for (size_t k = B.tid; k < pp; k += B.nt) A[k] = 0.0;
    __syncthreads();
    // Q(r, r2) = sum over the standard columns i of rows r, r2 of
    // A(r,i) A(r2,i) d_i^2, plus d^2 of row r's slack on the diagonal; thread
    // r writes only row r (entries (r2, r) of column r2), in a fixed order
    for (int r = B.tid; r < p; r += B.nt) {
        for (uint32_t e = W.rptr[r]; e < W.rptr[r + 1]; ++e) {
            const uint16_t ent = W.rowent[e];
            const int i = ent & kIdx;
            const double dd = W.d2[i];
            for (uint32_t k = W.cptr[i]; k < W.cptr[i + 1]; ++k) {
                const uint16_t ce = W.colent[k];
                const int r2 = ce & kIdx;
                A[(size_t)r2 * p + r] += ((ent ^ ce) & kNeg) ? -dd : dd;
            }
        }
        A[(size_t)r * p + r] += W.d2[n + r];
    }
    __syncthreads();
    for (int j = 1 + B.tid; j < p; j += B.nt) A[(size_t)j * p + j - 1] = A[(size_t)j * p + j];
    __syncthreads();
    const bool sweeper = B.warp == B.sw;
    for (int k0 = 0; k0 < p; k0 += kDB) {
        const int kb = min(kDB, p - k0);
        int bad = 0;
        if (sweeper) bad = chol_diag_block(A, p, k0, kb, B.lane);
        if (__syncthreads_or(bad)) return false;   // (same value in every thread)
        const int r0 = k0 + kDB;
        if (r0 >= p) break;
        // rows below: x = a L11^-T, one row per thread (kb = kDB here)
        for (int i = r0 + B.tid; i < p; i += B.nt) {
            double x[kDB];
#pragma unroll
            for (int t = 0; t < kDB; ++t) x[t] = A[(size_t)(k0 + t) * p + i];
#pragma unroll
            for (int t = 0; t < kDB; ++t) {
                const double* ct = A + (size_t)(k0 + t) * p + k0;   // column k0+t of the block
                double v = x[t];
#pragma unroll
                for (int s2 = 0; s2 < t; ++s2) v -= x[s2] * A[(size_t)(k0 + s2) * p + k0 + t];
                x[t] = v / ct[t];
            }
#pragma unroll
            for (int t = 0; t < kDB; ++t) A[(size_t)(k0 + t) * p + i] = x[t];
        }
        __syncthreads();
        // trailing lower triangle -= L21 L21', 4 x 4 tiles (bi >= bj),
        // enumerated column tile by column tile
        const int m2 = p - r0, nb4 = (m2 + 3) >> 2;
        const int ntile = nb4 * (nb4 + 1) / 2;
        for (int b = B.tid; b < ntile; b += B.nt) {
            // column tile bj: tiles bj..nb4-1, starting at off(bj) = bj nb4 - bj (bj - 1) / 2
            int bj = (int)((2.0 * nb4 + 1.0 - sqrt((2.0 * nb4 + 1.0) * (2.0 * nb4 + 1.0) - 8.0 * b)) * 0.5);
            bj = max(0, min(bj, nb4 - 1));
            while (bj > 0 && bj * nb4 - bj * (bj - 1) / 2 > b) --bj;
            while (bj + 1 < nb4 && (bj + 1) * nb4 - (bj + 1) * bj / 2 <= b) ++bj;
            const int bi = bj + (b - (bj * nb4 - bj * (bj - 1) / 2));
            const int i0 = r0 + 4 * bi, j0 = r0 + 4 * bj;
            double acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
#pragma unroll 4
            for (int t = 0; t < kDB; ++t) {
                const double* ct = A + (size_t)(k0 + t) * p;
                double li[4], lj[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    li[a] = i0 + a < p ? ct[i0 + a] : 0.0;
                    lj[a] = j0 + a < p ? ct[j0 + a] : 0.0;
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] = fma(li[a], lj[c], acc[a][c]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + c;
                if (j >= p) continue;
                double* cj = A + (size_t)j * p;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = i0 + a;
                    if (i < p && i >= j) cj[i] -= acc[a][c];
                }
            }
        }
        __syncthreads();
    }
    // L y = w (into r64), panel by panel
    for (int r = B.tid; r < p; r += B.nt) W.r64[r] = W.w[r];
    __syncthreads();
    for (int k0 = 0; k0 < p; k0 += kDB) {
        const int kb = min(kDB, p - k0);
        if (sweeper)
            for (int j = k0; j < k0 + kb; ++j) {
                const double* cj = A + (size_t)j * p;
                const double yj = W.r64[j] / cj[j];
                __syncwarp();
                const int i = j + 1 + B.lane;
                if (i < k0 + kb) W.r64[i] -= cj[i] * yj;
                if (B.lane == 0) W.r64[j] = yj;
                __syncwarp();
            }
        __syncthreads();
        for (int i = k0 + kb + B.tid; i < p; i += B.nt) {
            double v = W.r64[i];
            for (int t = 0; t < kb; ++t) v -= A[(size_t)(k0 + t) * p + i] * W.r64[k0 + t];
            W.r64[i] = v;
        }
        __syncthreads();
    }
    // L' dy = y, panel by panel from the last
    for (int r = B.tid; r < p; r += B.nt) W.dy[r] = W.r64[r];
    __syncthreads();
    for (int k0 = ((p - 1) / kDB) * kDB; k0 >= 0; k0 -= kDB) {
        const int kb = min(kDB, p - k0);
        if (sweeper)
            for (int j = k0 + kb - 1; j >= k0; --j) {
                const double* cj = A + (size_t)j * p;
                // dy_j = (y_j - sum_{j < i < k0+kb} L(i,j) dy_i) / L(j,j)
                const int i = j + 1 + B.lane;
                double part = i < k0 + kb ? cj[i] * W.dy[i] : 0.0;
                const double sum = warp_sum(part);
                __syncwarp();
                if (B.lane == 0) W.dy[j] = (W.dy[j] - sum) / cj[j];
                __syncwarp();
            }
        __syncthreads();
        // rows above the panel: dy_i -= sum_t L(k0+t, i) dy_{k0+t}
        for (int i = B.tid; i < k0; i += B.nt) {
            const double* ci = A + (size_t)i * p + k0;
            double v = W.dy[i];
            for (int t = 0; t < kb; ++t) v -= ci[t] * W.dy[k0 + t];
            W.dy[i] = v;
        }
        __syncthreads();
    }
    return true;
}

template <typename T>
__device__ inline NewtonOut newton_solve(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                         const Levels& L, const DevParams& P, double tol,
                                         int max_it, bool& force64, bool& force_dense) {
    const int p = F.p;
    double ww = 0.0;
    for (int r = B.tid; r < p; r += B.nt) { W.dy[r] = 0.0; W.r64[r] = W.w[r]; ww += W.w[r] * W.w[r]; }
    const double wn = sqrt(bsum(B, ww));
    NewtonOut o{0, 0, 0, 0.0, 0.0, 0.0};
    if (wn == 0.0) return o;
    const double it_flops = pcg_iter_flops(F, C.n, (int)(W.bptr[p] + W.fptr[p]));
    const int nnz_m = p + (int)W.bptr[p];
    double rn = wn;
    const bool dense_ok = W.qd != nullptr && F.p <= W.dense_p;
    if (force_dense && dense_ok && dense_newton<T>(B, C, W, F)) {   // PCG already failed in this LP
        double rr;
        residual64<double, T>(B, C, W, F, &rr);
        o.dense = 1;
        o.relres = sqrt(rr) / wn;
        o.flops += dense_flops(F, C.n);
        return o;
    }
    bool use64 = sizeof(T) == 8 || force64;
    // LPDEC_M32: FP32 M-solves until one round stalls, then FP64 M-solves
    // for the rest of this LP (force64 is sticky across its Newton solves)
    bool m32 = P.precision == LPDEC_M32 && !force64;
    bool view_ready = false;
    const int fp32_cap = max(64, max_it / 8);   // one FP32 round; failing it switches to FP64
    const int m32_cap = max(256, max_it / 4);   // one round with an FP32 M-solve
    WS<double> W64;
    for (int round = 0; round < 12; ++round) {
        if (rn < tol * wn || o.iters >= max_it) break;
        double target = tol * wn / rn;
        double rel = 0.0;
        int it;
        if (!use64) {
            target = fmax(target, P.tol_inner);
            it = refine_round<T, T>(B, C, W, W, F, L, rn, target, min(fp32_cap, max_it - o.iters),
                                    &rel);
        } else if (sizeof(T) == 8) {
            it = refine_round<T, T>(B, C, W, W, F, L, rn, target,
                                    m32 ? min(m32_cap, max_it - o.iters) : max_it - o.iters,
                                    &rel, m32);
            if (!m32) o.iters64 += it;
        } else {
            if (!view_ready) {
                W64 = fp64_view<T>(W);
                for (int r = B.tid; r < p; r += B.nt) W64.invd2p[r] = 1.0 / W.d2[W.pivcol[r]];
                __syncthreads();
                view_ready = true;
            }
            it = refine_round<double, T>(B, C, W64, W, F, L, rn, target, max_it - o.iters, &rel);
            o.iters64 += it;
        }
        o.iters += it;
        o.flops += it * it_flops + 4.0 * F.ea + C.n + 3.0 * p;
        o.bytes += it * pcg_iter_bytes(F, C.n, nnz_m, use64 ? 8 : (int)sizeof(T));
        double rr;
        residual64<double, T>(B, C, W, F, &rr);
        double rn_new = sqrt(rr);
        bool halved = rn_new < 0.5 * rn;
        bool missed = rel > target;   // PCG stopped at its budget
        rn = rn_new;
        if (!use64) {
            if (!halved || missed) use64 = force64 = true;   // FP64 from here on in this LP
        } else if (m32) {
            if (!halved || missed) { m32 = false; force64 = true; }
        } else if (!halved) {
            break;
        }
    }
    o.relres = rn / wn;
    // PCG that converged but ran long (lpdec_params.dense_switch): the later
    // Newton systems of this LP only get harder, so they go to the direct
    // solve, cheaper than that many PCG iterations. A dense solve costs
    // p^3/6 FMAs, a PCG iteration about p sequential steps: above 512 rows
    // the threshold grows as (p/512)^2 (below, fixed costs of both keep it
    // flat).
    if (dense_ok && P.dense_switch > 0 &&
        o.iters > P.dense_switch * fmax(1.0, ((double)p * p) / (512.0 * 512.0)))
        force_dense = true;
    if (o.relres > tol && dense_ok) {   // PCG stalled: direct solve, for the rest of the LP
        force_dense = true;
        if (dense_newton<T>(B, C, W, F)) {
            double rr;
            residual64<double, T>(B, C, W, F, &rr);
            o.dense = 1;
            o.relres = sqrt(rr) / wn;
            o.flops += dense_flops(F, C.n);
        }
    }
    return o;
}

// ---------------------------------------------------------------------------
// Optimality certificate. Section VI-A: the unique LP solution is strictly
// complementary, its basic set B = {i : x*_i > 0} has linearly independent
// columns, and near the optimum x_i > z_i exactly on B. Given the partition
// read from (x, z):
//   primal  x^_N = 0, A_B x^_B = b (minimum-norm correction of x_B by CGLS);
//   dual    y^ = y + A_B lam with (A_B' A_B) lam = c_B - A_B' y (CG), so that
//           z^_B = c_B - A_B' y^ = 0;
// and x^ >= 0, z^_N = c_N - A_N' y^ >= 0. Primal and dual feasibility with
// complementarity prove x^ optimal, and since the optimum is unique x^ is it,
// whatever the accuracy of the iterate it came from. On success x := x^.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double rowA_basic(const CodeView& C, const WS<T>& W, int r,
                                             const double* v) {
    double acc = 0.0;
    const uint32_t e1 = W.rptr[r + 1];
    for (uint32_t e = W.rptr[r]; e < e1; ++e) {
        uint16_t ent = W.rowent[e];
        int i = ent & kIdx;
        if (W.basic[i]) acc += signed_val<double>(ent, v[i]);
    }
    if (W.basic[C.n + r]) acc += v[C.n + r];
    return acc;
}
template <typename T>
__device__ __forceinline__ double colA_basic(const CodeView& C, const WS<T>& W, int i,
                                             const double* s) {
    if (!W.basic[i]) return 0.0;
    return i < C.n ? colA_T<double>(C, W, i, s) : s[i - C.n];
}

__device__ __forceinline__ double cost_of(const double* gamma, int n, int i) {
    return i < n ? fabs(gamma[i]) : 0.0;
}

template <typename T>
__device__ __noinline__ int certify(Blk& B, const CodeView C, WS<T> W, const Frame& F,
                              const double* gamma) {
    const int n = C.n, p = F.p, q = F.q;
    double nbasic = 0.0, cmax = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {
        uint8_t bi = W.x[i] > W.zz[i] ? 1 : 0;
        W.basic[i] = bi;
        nbasic += bi;
        W.v1[i] = 0.0;
        W.vx[i] = bi ? W.x[i] : 0.0;
        cmax = fmax(cmax, cost_of(gamma, n, i));
    }
    double2 nb = bsum2(B, nbasic, 0.0);
    cmax = -bmin2(B, -cmax, 0.0).x;
    const int max_it = 2 * (int)nb.x + 50;   // CG on the basis: at most its size in exact arithmetic
    // --- primal: CGLS on A_B d = s, s = b - A_B x_B
    double* d = W.v1; double* g = W.v2; double* h = W.v3; double* sr = W.vr1; double* lr = W.vr2;
    double ss = 0.0, bb = 0.0;
    for (int r = B.tid; r < p; r += B.nt) {
        double v = W.b[r] - rowA_basic(C, W, r, W.vx);
        sr[r] = v;
        ss += v * v;
        bb += W.b[r] * W.b[r];
    }
    double2 t0 = bsum2(B, ss, bb);
    ss = t0.x;
    const double pstop = 1e-13 * (1.0 + sqrt(t0.y));
    double gg = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {
        double v = colA_basic(C, W, i, sr);
        g[i] = v; h[i] = v; gg += v * v;
    }
    gg = bsum(B, gg);
    for (int it = 0; it < max_it && sqrt(ss) > pstop && gg > 0.0; ++it) {
        double ll = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            double v = rowA_basic(C, W, r, h);
            lr[r] = v; ll += v * v;
        }
        ll = bsum(B, ll);
        if (!(ll > 0.0)) break;
        const double a = gg / ll;
        for (int i = B.tid; i < q; i += B.nt) d[i] += a * h[i];
        double sl = 0.0;
        for (int r = B.tid; r < p; r += B.nt) { double v = sr[r] - a * lr[r]; sr[r] = v; sl += v * v; }
        ss = bsum(B, sl);
        double gl = 0.0;
        for (int i = B.tid; i < q; i += B.nt) { double v = colA_basic(C, W, i, sr); g[i] = v; gl += v * v; }
        const double gg2 = bsum(B, gl);
        const double beta = gg2 / gg;
        gg = gg2;
        for (int i = B.tid; i < q; i += B.nt) h[i] = g[i] + beta * h[i];
        __syncthreads();
    }
    double mnx = INFINITY;
    for (int i = B.tid; i < q; i += B.nt) {
        double v = W.basic[i] ? W.vx[i] + d[i] : 0.0;
        W.vx[i] = v;
        if (W.basic[i]) mnx = fmin(mnx, v);
    }
    __syncthreads();
    double res = 0.0;
    for (int r = B.tid; r < p; r += B.nt)
        res = fmax(res, fabs(rowA<double>(C, W, r, W.vx) + W.vx[n + r] - W.b[r]));
    double2 pm = bmin2(B, mnx, -res);
    if (!(pm.x >= -1e-11 && -pm.y <= 1e-9)) return 0;
    // --- dual: CG on (A_B' A_B) lam = t, t = c_B - A_B' y
    double* lam = W.v1; double* rq = W.v2; double* pq = W.v3; double* kq = W.v4;
    double* ap = W.vr1; double* yh = W.vr2;
    double rr = 0.0, tt = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {
        double v = 0.0;
        if (W.basic[i]) {
            double aty = (i < n) ? colA_T<double>(C, W, i, W.y) : W.y[i - n];
            v = cost_of(gamma, n, i) - aty;
        }
        lam[i] = 0.0; rq[i] = v; pq[i] = v; rr += v * v;
        tt += cost_of(gamma, n, i) * cost_of(gamma, n, i);
    }
    double2 t1 = bsum2(B, rr, tt);
    rr = t1.x;
    const double dstop = 1e-13 * (1.0 + sqrt(t1.y));
    for (int it = 0; it < max_it && sqrt(rr) > dstop; ++it) {
        for (int r = B.tid; r < p; r += B.nt) ap[r] = rowA_basic(C, W, r, pq);
        __syncthreads();
        double pkp = 0.0;
        for (int i = B.tid; i < q; i += B.nt) { double v = colA_basic(C, W, i, ap); kq[i] = v; pkp += pq[i] * v; }
        pkp = bsum(B, pkp);
        if (!(pkp > 0.0)) break;
        const double a = rr / pkp;
        double rl = 0.0;
        for (int i = B.tid; i < q; i += B.nt) {
            lam[i] += a * pq[i];
            double v = rq[i] - a * kq[i];
            rq[i] = v; rl += v * v;
        }
        const double rr2 = bsum(B, rl);
        const double beta = rr2 / rr;
        rr = rr2;
        for (int i = B.tid; i < q; i += B.nt) pq[i] = rq[i] + beta * pq[i];
        __syncthreads();
    }
    for (int r = B.tid; r < p; r += B.nt) yh[r] = W.y[r] + rowA_basic(C, W, r, lam);
    __syncthreads();
    double zmin_n = INFINITY, zmax_b = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {
        double aty = (i < n) ? colA_T<double>(C, W, i, yh) : yh[i - n];
        double zi = cost_of(gamma, n, i) - aty;
        if (W.basic[i]) zmax_b = fmax(zmax_b, fabs(zi));
        else zmin_n = fmin(zmin_n, zi);
    }
    double2 dm = bmin2(B, zmin_n, -zmax_b);
    const double scale = 1.0 + cmax;
    if (!(dm.x >= -1e-11 * scale && -dm.y <= 1e-8 * scale)) return 0;
    for (int i = B.tid; i < q; i += B.nt) W.x[i] = W.vx[i];
    __syncthreads();
    return 1;
}

// Certificate from the MTS basis. The p selected columns M form a
// nonsingular (triangular) basis of A. Near the optimum of an integral LP
// they contain the basic set B, and then
//   x_M = A_M^-1 b  (one back substitution)
// is the optimal vertex. The dual is pinned to the iterate's partition:
// z^_i = 0 for basic i in M, z^_i = c_i - (A'y)_i for the other columns of
// M, and A_M' y^ = c_M - z^_M (one forward substitution). If x^ >= 0,
// z^ = c - A'y^ >= 0 on every column and x^_i z^_i = 0, the pair is primal
// and dual feasible and complementary, so x^ is optimal (and, the optimum
// being unique, the vertex the oracle reaches). On success x := x^.
template <typename T>
__device__ __noinline__ int certify_basis(Blk& B, const CodeView C, WS<T> W, const Frame& F,
                                    const Levels& L, const double* gamma) {
    const int n = C.n, p = F.p, q = F.q;
    WS<double> D = fp64_view<T>(W);
    double* rhs = W.vr1;
    double* out = W.vr2;
    double cmax = 0.0;
    for (int r = B.tid; r < p; r += B.nt) rhs[r] = W.b[r];
    for (int i = B.tid; i < q; i += B.nt) cmax = fmax(cmax, cost_of(gamma, n, i));
    __syncthreads();
    level_sweep<double, true>(B, D, W.lbptr, W.lbrows, W.lbse, L.nb, rhs, out, 0.0);
    // x^ over the columns (pivot column of row r gets out[r])
    double mnx = INFINITY;
    for (int i = B.tid; i < q; i += B.nt) W.vx[i] = 0.0;
    __syncthreads();
    for (int r = B.tid; r < p; r += B.nt) {
        double v = out[r];
        W.vx[W.pivcol[r]] = v;
        mnx = fmin(mnx, v);
    }
    // right side of A_M' y^ = c_M - z^_M, indexed by the pivot row
    for (int r = B.tid; r < p; r += B.nt) {
        int i = W.pivcol[r];
        double c = cost_of(gamma, n, i);
        double zt = 0.0;
        if (!(W.x[i] > W.zz[i])) zt = c - ((i < n) ? colA_T<double>(C, W, i, W.y) : W.y[i - n]);
        out[r] = c - zt;
    }
    double2 m0 = bmin2(B, mnx, -cmax);
    cmax = -m0.y;
    const double tol = 1e-11 * (1.0 + cmax);
    if (!(m0.x >= -tol)) return 0;
    level_sweep<double, false, false>(B, D, W.lfptr, W.lfrows, W.lfse, L.nf, rhs, out, 0.0);
    double zmin = INFINITY, comp = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {
        double aty = (i < n) ? colA_T<double>(C, W, i, out) : out[i - n];
        double zi = cost_of(gamma, n, i) - aty;
        zmin = fmin(zmin, zi);
        comp = fmax(comp, fabs(W.vx[i] * zi));
    }
    double2 m1 = bmin2(B, zmin, -comp);
    if (!(m1.x >= -tol && -m1.y <= tol)) return 0;
    for (int i = B.tid; i < q; i += B.nt) W.x[i] = fmax(W.vx[i], 0.0);
    __syncthreads();
    return 1;
}

// ---------------------------------------------------------------------------
// a3 + a6: infeasible primal-dual path-following method (Section IV-B)
// ---------------------------------------------------------------------------
// Doubles per interior-point iteration in a trace (lpdec_lp_solve_trace_device).
constexpr int kTrace = 10;
// Least x_i, z_i of a warm start (lpdec_params.warm_start).
constexpr double kWarmFloor = 1e-2;

struct IpmOut {
    int iters, pcg_iters, pcg_iters64, converged, certified, max_levels, dense;
    double flops, bytes;
    double t_mts, t_pcg, t_dense, t_cert;   // phase times (s), lpdec_stats.sec_*
};

// trace (optional): per iteration 8 doubles {gap, feas_p, feas_d, PCG
// iterations, Newton relative residual, beta_P, beta_D, levels}
template <typename T>
__device__ __noinline__ IpmOut ipm_solve(Blk& B, const CodeView C, WS<T> W, Frame& F,
                                   const DevParams& P, const double* gamma, int q2,
                                   double* trace = nullptr, int max_trace = 0, bool warm = false) {
    const int n = C.n, p = F.p, q = F.q;
    IpmOut o{0, 0, 0, 0, 0, 0, 0, 0.0, 0.0};
    double nc2 = 0.0;
    if (!warm) {
        // cold start x = e, y = 0, z = c + e
        for (int i = B.tid; i < q; i += B.nt) {
            double c = cost_of(gamma, n, i);
            W.x[i] = 1.0;
            W.zz[i] = c + 1.0;
            nc2 += c * c;
        }
        for (int r = B.tid; r < p; r += B.nt) W.y[r] = 0.0;
    } else {
        // warm start from the previous LP's final iterate, pushed kWarmFloor
        // away from the boundary; a row kept from it (same check and set)
        // keeps its slack pair and dual, a new row starts as in a cold start
        for (int i = B.tid; i < n; i += B.nt) {
            double c = cost_of(gamma, n, i);
            W.x[i] = fmax(W.xw[i], kWarmFloor);
            W.zz[i] = fmax(W.zw[i], kWarmFloor);
            nc2 += c * c;
        }
        for (int r = B.tid; r < p; r += B.nt) {
            const int j = W.cchk[r], pr = W.prow[j];
            const bool kept = pr >= 0 && W.pmask[j] == W.cmask[r];
            W.x[n + r] = kept ? fmax(W.xw[n + pr], kWarmFloor) : 1.0;
            W.zz[n + r] = kept ? fmax(W.zw[n + pr], kWarmFloor) : 1.0;
            W.y[r] = kept ? W.yw[pr] : 0.0;
        }
    }
    F.normc = sqrt(bsum(B, nc2));   // (barrier inside)
    bool force64 = false, force_dense = false;
    int last_pcg = 0;
    // preconditioner of this LP's Newton systems (LPDEC_MTS_ADAPTIVE starts
    // column-wise and turns incremental for good after a long PCG run)
    int kind = P.precond == LPDEC_MTS_ADAPTIVE ? LPDEC_MTS_COLUMN : P.precond;
    Levels L{0, 0};
    bool reuse_ok = false;
    double nbasic_prev = -1.0;
    double prev_grel = INFINITY, sig0 = -1.0, sig1 = -1.0;
    for (int it = 0;; ++it) {
        if (P.abort && (it & 3) == 3 && aborted(P)) { o.iters = it; break; }
        // Expensive regime (the basis certificate keeps failing and Newton
        // solves need hundreds of PCG iterations, typical of LPs with a
        // fractional optimum): below gap tol_cert, whenever the partition
        // x_i > z_i has not moved for an iteration, try the general
        // certificate (CG on the basic columns), far cheaper than one more
        // interior-point iteration here.
        if (prev_grel < P.tol_cert && last_pcg > 200) {
            double c0 = 0.0, c1 = 0.0;
            for (int i = B.tid; i < q; i += B.nt)
                if (W.x[i] > W.zz[i]) { c0 += 1.0; c1 += (double)(i + 1) * (double)(i + 1); }
            double2 sg = bsum2(B, c0, c1);
            if (sg.x == sig0 && sg.y == sig1) {
                const unsigned long long tc = global_ns();
                const int okc = certify<T>(B, C, W, F, gamma);
                o.t_cert += since(tc);
                if (okc) {
                    o.converged = 1;
                    o.certified = 1;
                    o.iters = it;
                    break;
                }
            }
            sig0 = sg.x;
            sig1 = sg.y;
        }
        // residuals r_b = b - A x (into W.w), r_c = c - A'y - z (into W.rc)
        double nrb2 = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            double v = W.b[r] - (rowA<double>(C, W, r, W.x) + W.x[n + r]);
            W.w[r] = v;
            nrb2 += v * v;
        }
        double nrc2 = 0.0, gap = 0.0, cx = 0.0;
        for (int i = B.tid; i < q; i += B.nt) {
            double aty = (i < n) ? colA_T<double>(C, W, i, W.y) : W.y[i - n];
            double c = cost_of(gamma, n, i);
            double v = c - aty - W.zz[i];
            W.rc[i] = v;
            nrc2 += v * v;
            gap += W.x[i] * W.zz[i];
            cx += c * W.x[i];
        }
        double2 s1 = bsum2(B, nrb2, nrc2);
        double2 s2 = bsum2(B, gap, cx);
        gap = s2.x;
        cx = s2.y;
        const double g_rel = gap / (1.0 + fabs(cx));
        const double fp = sqrt(s1.x) / (1.0 + F.normb);
        const double fd = sqrt(s1.y) / (1.0 + F.normc);
        if (g_rel < P.tol_gap && ((fp < P.tol_feas && fd < P.tol_feas) ||
                                  (fp < P.tol_feas_loose && fd < P.tol_feas_loose))) {
            o.converged = 1;
            o.iters = it;
            break;
        }
        if (it == P.max_ipm) { o.iters = it; break; }
        const double mu = P.sigma * gap / (double)q;
        // D^2 = X Z^-1 (Eq. 27); W.rc := D^2 r_c - Z^-1 r_e over the columns
        for (int i = B.tid; i < q; i += B.nt) {
            double xi = W.x[i], zi = W.zz[i];
            double d2 = xi / zi;
            double re = mu - xi * zi;
            W.d2[i] = d2;
            W.rc[i] = d2 * W.rc[i] - re / zi;
        }
        __syncthreads();
        // w = r_b + A D^2 r_c - A Z^-1 r_e (Eq. 24 right side)
        for (int r = B.tid; r < p; r += B.nt) W.w[r] += rowA<double>(C, W, r, W.rc) + W.rc[n + r];
        __syncthreads();
        // MTS reuse (lpdec_params.mts_reuse): keep the previous iteration's
        // triangular set while its PCG converged fast and the partition
        // x_i > z_i kept its size; the values of M (D_M^2) are always current
        unsigned long long tp = global_ns();
        if (!(P.mts_reuse && reuse_ok)) L = select_mts<T>(B, C, W, F, W.d2, kind);
        o.t_mts += since(tp);
        o.max_levels = max(o.max_levels, max(L.nb, L.nf));
        // near the optimum the selected basis may already be optimal
        if (g_rel < P.tol_cert) {
            tp = global_ns();
            const int okb = certify_basis<T>(B, C, W, F, L, gamma);
            o.t_cert += since(tp);
            if (okb) {
                o.converged = 1;
                o.certified = 1;
                o.iters = it;
                break;
            }
        }
        for (int i = B.tid; i < q; i += B.nt) W.d2t[i] = (T)W.d2[i];
        for (int r = B.tid; r < p; r += B.nt) {
            int pc = W.pivcol[r];
            W.invd2p[r] = pc < q ? (T)(1.0 / W.d2[pc]) : T(0);
            if (P.precision == LPDEC_M32) W.ip32[r] = pc < q ? (float)(1.0 / W.d2[pc]) : 0.0f;
        }
        __syncthreads();
        const double tol = fmax(P.tol_pcg, fmin(1e-3, P.pcg_gap_factor * g_rel));
        if (W.lz && B.tid == 0) { W.lz[2 * kLz] = 0.0; W.lz[2 * kLz + 1] = 0.0; }
        __syncthreads();
        tp = global_ns();
        NewtonOut no = newton_solve<T>(B, C, W, F, L, P, tol, P.max_pcg, force64, force_dense);
        if (no.dense) o.t_dense += since(tp);
        else o.t_pcg += since(tp);
        o.dense += no.dense;
        o.pcg_iters += no.iters;
        o.pcg_iters64 += no.iters64;
        o.flops += no.flops;
        o.bytes += no.bytes;
        last_pcg = no.dense ? 1000000 : no.iters;
        if (P.mts_reuse) {
            double nb_l = 0.0;
            for (int i = B.tid; i < q; i += B.nt) nb_l += W.x[i] > W.zz[i] ? 1.0 : 0.0;
            const double nbasic = bsum(B, nb_l);
            reuse_ok = last_pcg <= 20 && nbasic == nbasic_prev;
            nbasic_prev = nbasic;
        }
        if (P.precond == LPDEC_MTS_ADAPTIVE && (no.dense || no.iters > P.precond_switch))
            kind = LPDEC_MTS_INCREMENTAL;
        if (no.relres > 1e-3 && g_rel < 1e-6) {   // no usable direction left near the optimum
            o.iters = it;
            break;
        }
        // Newton direction (Eqs. 25-26), with r_c recomputed from (x, y, z)
        double ap = INFINITY, ad = INFINITY;
        for (int i = B.tid; i < q; i += B.nt) {
            double xi = W.x[i], zi = W.zz[i];
            double d2 = W.d2[i];
            double re = mu - xi * zi;
            double aty = (i < n) ? colA_T<double>(C, W, i, W.y) : W.y[i - n];
            double rc = cost_of(gamma, n, i) - aty - zi;
            double atdy = (i < n) ? colA_T<double>(C, W, i, W.dy) : W.dy[i - n];
            double dx = d2 * (atdy - rc) + re / zi;
            double dz = (re - zi * dx) / xi;
            W.rc[i] = dx;
            W.d2[i] = dz;
            if (dx < 0.0) ap = fmin(ap, -xi / dx);
            if (dz < 0.0) ad = fmin(ad, -zi / dz);
        }
        double2 mn = bmin2(B, ap, ad);
        const double bp = fmin(1.0, P.eta * mn.x);
        const double bd = fmin(1.0, P.eta * mn.y);
        if (trace && it < max_trace && B.tid == 0) {
            double* tr = trace + kTrace * it;
            tr[0] = g_rel; tr[1] = fp; tr[2] = fd; tr[3] = no.iters; tr[4] = no.relres;
            tr[5] = bp; tr[6] = bd; tr[7] = max(L.nb, L.nf);
            tr[8] = tr[9] = NAN;
            if (W.lz) lz_extremes(W.lz, &tr[8], &tr[9]);
        }
        for (int i = B.tid; i < q; i += B.nt) {
            W.x[i] += bp * W.rc[i];
            W.zz[i] += bd * W.d2[i];
        }
        for (int r = B.tid; r < p; r += B.nt) W.y[r] += bd * W.dy[r];
        __syncthreads();
        prev_grel = g_rel;
    }
    return o;
}

// ---------------------------------------------------------------------------
// Optimal vertex from the final iterate (partition basic iff x_i > z_i,
// Section VI-A): x_N = 0 and A_B x_B = b, solved as the minimum-norm
// correction d of x_B by CGLS in FP64. Accepted when the vertex is primal
// feasible to 1e-9 and its cost is within 1e-6 of the iterate's; otherwise
// only x_N is zeroed. Vectors: d and g over columns (W.rc, W.d2), the search
// direction h over columns (standard part W.t64, slack part W.dy), s and l
// over rows (W.w, W.r64).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int vertex_recover(Blk& B, const CodeView C, WS<T> W, const Frame& F,
                                     const double* gamma) {
    const int n = C.n, p = F.p, q = F.q;
    double* d = W.rc;
    double* g = W.d2;
    double* hs = W.t64;
    double* hk = W.dy;
    double* s = W.w;
    double* lr = W.r64;
    for (int i = B.tid; i < q; i += B.nt) {
        W.basic[i] = W.x[i] > W.zz[i] ? 1 : 0;
        d[i] = 0.0;
    }
    __syncthreads();
    double ss = 0.0, nb_ = 0.0;
    for (int r = B.tid; r < p; r += B.nt) {   // s = b - A_B x_B
        double acc = 0.0;
        for (uint32_t e = W.rptr[r]; e < W.rptr[r + 1]; ++e) {
            uint16_t ent = W.rowent[e];
            int i = ent & kIdx;
            if (W.basic[i]) acc += signed_val<double>(ent, W.x[i]);
        }
        if (W.basic[n + r]) acc += W.x[n + r];
        double v = W.b[r] - acc;
        s[r] = v;
        ss += v * v;
        nb_ += W.b[r] * W.b[r];
    }
    double2 t0 = bsum2(B, ss, nb_);
    ss = t0.x;
    const double stop = 1e-13 * (1.0 + sqrt(t0.y));
    double gg = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {   // g = A_B' s, h = g
        double v = 0.0;
        if (W.basic[i]) v = (i < n) ? colA_T<double>(C, W, i, s) : s[i - n];
        g[i] = v;
        if (i < n) hs[i] = v; else hk[i - n] = v;
        gg += v * v;
    }
    gg = bsum(B, gg);
    const int max_it = 2 * p + 50;
    for (int it = 0; it < max_it && sqrt(ss) > stop && gg > 0.0; ++it) {
        double ll = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            double v = rowA<double>(C, W, r, hs) + hk[r];
            lr[r] = v;
            ll += v * v;
        }
        ll = bsum(B, ll);
        if (!(ll > 0.0)) break;
        double a = gg / ll;
        for (int i = B.tid; i < q; i += B.nt) d[i] += a * ((i < n) ? hs[i] : hk[i - n]);
        double ss_l = 0.0;
        for (int r = B.tid; r < p; r += B.nt) { double v = s[r] - a * lr[r]; s[r] = v; ss_l += v * v; }
        ss = bsum(B, ss_l);
        double gg_l = 0.0;
        for (int i = B.tid; i < q; i += B.nt) {
            double v = 0.0;
            if (W.basic[i]) v = (i < n) ? colA_T<double>(C, W, i, s) : s[i - n];
            g[i] = v;
            gg_l += v * v;
        }
        double gg2 = bsum(B, gg_l);
        double beta = gg2 / gg;
        gg = gg2;
        for (int i = B.tid; i < q; i += B.nt) {
            if (i < n) hs[i] = g[i] + beta * hs[i];
            else hk[i - n] = g[i] + beta * hk[i - n];
        }
        __syncthreads();
    }
    // candidate vertex (into g) and its checks
    double mnx = INFINITY, c_new = 0.0, c_old = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {
        double v = W.basic[i] ? W.x[i] + d[i] : 0.0;
        g[i] = v;
        if (W.basic[i]) mnx = fmin(mnx, v);
        double c = cost_of(gamma, n, i);
        c_new += c * v;
        c_old += c * W.x[i];
    }
    __syncthreads();
    double res = 0.0;
    for (int r = B.tid; r < p; r += B.nt)
        res = fmax(res, fabs(rowA<double>(C, W, r, g) + g[n + r] - W.b[r]));
    double2 m1 = bmin2(B, mnx, -res);
    double2 cs = bsum2(B, c_new, c_old);
    bool ok = m1.x >= -1e-9 && (-m1.y) <= 1e-9 && fabs(cs.x - cs.y) <= 1e-6 * (1.0 + fabs(cs.y));
    for (int i = B.tid; i < q; i += B.nt) {
        if (ok) W.x[i] = g[i];
        else if (!W.basic[i]) W.x[i] = 0.0;
    }
    __syncthreads();
    return ok ? 0 : 1;
}

// One LP of the adaptive loop: the interior-point method, then its vertex
// with an optimality certificate. An iterate that has not separated the
// optimal partition yet (the certificate fails although the method
// converged) is refined by solving again at a 100x, then 1000x tighter gap
// (twice the iteration cap); only if that fails too is the partition's
// vertex taken without a certificate (counted in vertex_failures). Returns
// whether the LP ended converged or certified; io accumulates the counts.
// Keeps the final iterate of the LP just solved (before its vertex replaces
// x) for the warm start of the next LP: x, z over the columns, y over the
// rows, and per check its row and set.
template <typename T>
__device__ inline void save_iterate(Blk& B, const CodeView& C, WS<T>& W, const Frame& F) {
    for (int i = B.tid; i < F.q; i += B.nt) { W.xw[i] = W.x[i]; W.zw[i] = W.zz[i]; }
    for (int j = B.tid; j < C.m; j += B.nt) W.prow[j] = -1;
    __syncthreads();
    for (int r = B.tid; r < F.p; r += B.nt) {
        W.yw[r] = W.y[r];
        W.prow[W.cchk[r]] = r;
        W.pmask[W.cchk[r]] = W.cmask[r];
    }
    __syncthreads();
}

template <typename T>
__device__ inline bool solve_lp(Blk& B, const CodeView& C, WS<T>& W, Frame& F,
                                const DevParams& P, const double* gamma, lpdec_stats& st,
                                IpmOut& io, bool warm = false, bool keep = false) {
    io = ipm_solve<T>(B, C, W, F, P, gamma, 0, nullptr, 0, warm);
    if (keep) save_iterate<T>(B, C, W, F);
    unsigned long long tc = global_ns();
    int ok = io.certified || certify<T>(B, C, W, F, gamma);
    io.t_cert += since(tc);
    DevParams Q = P;
    Q.max_ipm = 2 * P.max_ipm;
    const unsigned long long tr = global_ns();
    for (int k = 0; k < 2 && !ok && io.converged; ++k) {
        Q.tol_gap = P.tol_gap * (k == 0 ? 1e-2 : 1e-3);
        IpmOut o2 = ipm_solve<T>(B, C, W, F, Q, gamma, 0);
        st.ipm_iters_refine += o2.iters;
        o2.iters += io.iters;
        o2.pcg_iters += io.pcg_iters;
        o2.pcg_iters64 += io.pcg_iters64;
        o2.dense += io.dense;
        o2.flops += io.flops;
        o2.bytes += io.bytes;
        o2.t_mts += io.t_mts;
        o2.t_pcg += io.t_pcg;
        o2.t_dense += io.t_dense;
        o2.t_cert += io.t_cert;
        o2.max_levels = max(o2.max_levels, io.max_levels);
        io = o2;
        tc = global_ns();
        ok = io.certified || certify<T>(B, C, W, F, gamma);
        io.t_cert += since(tc);
        if (ok || k == 1 || !io.converged) st.sec_refine += since(tr);
    }
    if (!ok) {
        tc = global_ns();
        st.vertex_failures += vertex_recover<T>(B, C, W, F, gamma);
        io.t_cert += since(tc);
    }
    return io.converged || ok;
}

// u from x (undo the flip of Eq. 16) and the active flags of the LP rows.
template <typename T>
__device__ inline void lp_finish(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                 const DevParams& P) {
    for (int i = B.tid; i < C.n; i += B.nt) W.u[i] = flipped(W.flip, i) ? 1.0 - W.x[i] : W.x[i];
    for (int r = B.tid; r < F.p; r += B.nt) W.cact[r] = (W.x[C.n + r] <= P.tau_act) ? 1 : 0;
    __syncthreads();
    for (int j = B.tid; j < C.m; j += B.nt) {
        uint8_t f = 0;
        for (uint32_t r = W.crptr[j]; r < W.crptr[j + 1]; ++r) f |= W.cact[r] ? kActive : 0;
        if (W.crptr[j + 1] > W.crptr[j]) W.flags[j] = kInLP | f;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Whole frame: MALP-A / MALP-B (Algorithm 3) driving a1..a6, then a7.
// ---------------------------------------------------------------------------
struct FrameOut {
    double* u;
    uint8_t* hard;
    int32_t* cert;
    uint32_t* mask;     // may be null
    lpdec_stats* stats; // may be null
};

// gamma'u over the frame (the same value in every thread).
template <typename T>
__device__ inline double frame_cost(Blk& B, const CodeView& C, WS<T>& W, const double* gamma) {
    double a = 0.0;
    for (int i = B.tid; i < C.n; i += B.nt) a += gamma[i] * W.u[i];
    return bsum(B, a);
}

// Moves a frame's cut list to the wide workspace (Lw, at gw): the row-sized
// arrays are re-pointed there, the list itself (rows and masks) copied.
template <typename T>
__device__ inline void widen(Blk& B, WS<T>& W, const Layout& Lw, char* gw, int p) {
    uint16_t* cchk = W.cchk;
    uint32_t* cmask = W.cmask;
    point_ws<T>(W, Lw, nullptr, gw, true);
    for (int r = B.tid; r < p; r += B.nt) { W.cchk[r] = cchk[r]; W.cmask[r] = cmask[r]; }
    __syncthreads();
}

template <typename T>
__device__ inline void decode_frame(Blk& B, const CodeView& C, const WS<T>& W0,
                                    const DevParams& P, const double* gamma, FrameOut out,
                                    int q2, int* shscan, const Layout* Lw = nullptr,
                                    char* gw = nullptr) {
    WS<T> W = W0;   // (the wide workspace, if this frame moves there, is its own)
    bool wide = false;
    const unsigned long long t0 = global_ns();
    int bad = 0;
    for (int i = B.tid; i < C.n; i += B.nt) bad |= !isfinite(gamma[i]);
    bad = __syncthreads_or(bad);
    Frame F{0, C.n, 0.0, 0.0, 0};
    lpdec_stats st{};
    st.t_start = (double)t0;
    if (bad) {
        st.status = LPDEC_ERR_INVALID_ARG;
        for (int i = B.tid; i < C.n; i += B.nt) { out.u[i] = NAN; out.hard[i] = 0; }
        if (out.mask) for (int j = B.tid; j < C.m; j += B.nt) out.mask[j] = 0;
        if (B.tid == 0) {
            *out.cert = 0;
            st.t_end = (double)global_ns();
            if (out.stats) *out.stats = st;
        }
        __syncthreads();
        return;
    }
    frame_init<T>(B, C, W, gamma);
    int status = LPDEC_OK;
    double cost = frame_cost(B, C, W, gamma);    // gamma'u^0
    bool alp = P.variant == LPDEC_ALP;           // Algorithm 1 semantics
    for (;;) {
        if (P.variant == LPDEC_MALP_B && !alp) drop_inactive<T>(B, C, W);
        if (P.abort && aborted(P)) { status = LPDEC_ERR_CANCELLED; break; }
        int added = cut_search<T>(B, C, W, P, alp);
        if (!added) break;
        if (st.alp_iters >= P.max_alp) { status = LPDEC_ERR_NOT_CONVERGED; break; }
        bool built = lp_build<T>(B, C, W, F, shscan, alp, wide ? C.pwide : C.pmax,
                                 wide ? C.eawide : C.eamax);
        if (!built && !wide && Lw && C.pwide > C.pmax) {
            widen<T>(B, W, *Lw, gw, F.p);
            wide = true;
            built = lp_build<T>(B, C, W, F, shscan, alp, C.pwide, C.eawide);
        }
        if (!built) { status = LPDEC_ERR_OUT_OF_BUDGET; break; }
        IpmOut io;
        // warm start (lpdec_params.warm_start) for MALP frames: one row per
        // check, so rows are matched by check and set
        const bool ws = P.warm_start && !alp;
        const bool solved = solve_lp<T>(B, C, W, F, P, gamma, st, io, ws && st.alp_iters > 0, ws);
        st.alp_iters++;
        st.ipm_iters_total += io.iters;
        st.pcg_iters_total += io.pcg_iters;
        st.pcg_iters_fp64 += io.pcg_iters64;
        st.dense_solves += io.dense;
        st.pcg_flops += io.flops;
        st.pcg_bytes += io.bytes;
        st.sec_mts += io.t_mts;
        st.sec_pcg += io.t_pcg;
        st.sec_dense += io.t_dense;
        st.sec_certify += io.t_cert;
        st.max_levels = max(st.max_levels, io.max_levels);
        lp_finish<T>(B, C, W, F, P);
        st.lp_rows_final = F.p;
        st.lp_rows_max = max(st.lp_rows_max, F.p);
        if (!solved) {
            status = P.abort && aborted(P) ? LPDEC_ERR_CANCELLED : LPDEC_ERR_NOT_CONVERGED;
            break;
        }
        // Theorem 2(b): with unique LP optima the MALP cost rises strictly. A
        // cost that does not rise means that hypothesis failed and MALP may
        // cycle between cut sets short of the optimum; the frame continues as
        // ALP (Algorithm 1), which only adds inequalities and reaches the LP
        // decoding optimum (Theorem 2(c)).
        const double next = frame_cost(B, C, W, gamma);
        if (!alp && next - cost <= P.tau_inc * (1.0 + fabs(cost))) {
            alp = true;
            st.alp_switch = st.alp_iters;
        }
        cost = next;
    }
    // a7: outputs. cert = integral; hard_i = [u_i > 1/2], the channel's
    // decision where u_i is within tau_int of 1/2. mask[j] = V of check j's
    // latest inequality.
    int frac = 0;
    double obj = 0.0;
    for (int i = B.tid; i < C.n; i += B.nt) {
        double ui = W.u[i];
        frac |= fabs(ui - rint(ui)) > P.tau_int;
        uint8_t hd = ui > 0.5 ? 1 : 0;
        if (fabs(ui - 0.5) <= P.tau_int) hd = gamma[i] < 0.0 ? 1 : 0;
        out.u[i] = ui;
        out.hard[i] = hd;
        obj += gamma[i] * ui;
    }
    if (out.mask)
        for (int j = B.tid; j < C.m; j += B.nt) out.mask[j] = (W.flags[j] & kInLP) ? W.mask[j] : 0u;
    frac = __syncthreads_or(frac);
    obj = bsum(B, obj);
    if (B.tid == 0) {
        *out.cert = frac ? 0 : 1;
        st.status = status;
        st.objective = obj;
        const unsigned long long t1 = global_ns();
        st.seconds = 1e-9 * (double)(t1 - t0);
        st.t_end = (double)t1;
        if (out.stats) *out.stats = st;
    }
    __syncthreads();
}

}  // namespace lpdec
