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
constexpr uint8_t kInLP = 1;     // check j has a parity inequality in the LP
constexpr uint8_t kActive = 2;   // ... and it is active at the last LP solution
constexpr uint16_t kNone = 0xffffu;
constexpr uint16_t kNeg = 0x8000u;   // packed entry: index | kNeg if the coefficient is -1
constexpr uint16_t kIdx = 0x7fffu;

// ---------------------------------------------------------------------------
// Code (H) view: CSR rows = checks, CSC columns = bits. Read-only, shared by
// every frame of a batch (n, m <= 32767).
// ---------------------------------------------------------------------------
struct CodeView {
    int n, m, E;
    const int* __restrict__ h_ptr;   // [m+1]
    const int* __restrict__ h_col;   // [E] bit of CSR edge e
    const int* __restrict__ e_chk;   // [E] check of CSR edge e
    const int* __restrict__ v_ptr;   // [n+1]
    const int* __restrict__ v_chk;   // [E] check of the k-th CSC entry
    const int* __restrict__ v_eidx;  // [E] CSR edge index of the k-th CSC entry
};

struct DevParams {
    double sigma, eta, tol_gap, tol_feas, tol_pcg, tau_act, tau_cut, tau_int;
    double pcg_gap_factor, tol_inner, tol_feas_loose;
    int max_alp, max_ipm, max_pcg, variant, precision;
};

// ---------------------------------------------------------------------------
// Workspace layout (the host decides shared vs global placement)
// ---------------------------------------------------------------------------
enum Arr {
    // hot arrays (shared memory)
    S_ROWENT, S_COLENT, S_ROWCHK, S_CHKROW, S_PIVCOL, S_PIVROW, S_PSGN,
    S_LB, S_LF, S_LBPTR, S_LFPTR, S_CUR, S_LBROWS, S_LFROWS, S_SELROW,
    S_DEG, S_BITMAP, S_FLAGS, S_MASK, S_FLIP,
    S_VEC,      // PCG vectors of type T: xs, r, z, h, l (m each), t (n), d2t (n+m), invd2p (m);
                // during the MTS selection the same bytes hold the u64 sort keys
                // [q2] followed by rank [q] and sorted [q] (uint16)
    // FP64 interior-point state (global scratch)
    G_X, G_Z, G_RC, G_D2, G_Y, G_B, G_W, G_DY, G_R64, G_U, G_T64, G_BASIC,
    A_COUNT
};

constexpr uint32_t kGlobalBit = 0x80000000u;

// Elements of type T in the S_VEC block: xs, r, z, h, l (m each), t (n),
// d2t (n + m), invd2p (m).
__host__ __device__ constexpr size_t vec_elems(int n, int m) {
    return 7 * (size_t)m + 2 * (size_t)n;
}

struct Layout {
    uint32_t off[A_COUNT];     // byte offset; kGlobalBit set = global scratch
    uint32_t smem_bytes;       // dynamic shared memory per CTA
    uint32_t q2;               // power of two >= n + m (sort width)
    unsigned long long gbytes; // global scratch bytes per CTA
};

template <typename T>
struct WS {
    uint16_t *rowent, *colent, *rowchk, *chkrow, *pivcol, *pivrow, *lb, *lf, *lbrows, *lfrows;
    uint16_t *selrow, *rank, *sorted;
    uint32_t *lbptr, *lfptr, *cur, *bitmap, *mask, *flip;
    uint8_t *psgn, *deg, *flags, *basic;
    T *xs, *r, *z, *h, *l, *t, *d2t, *invd2p;
    unsigned long long* skey;   // aliases the PCG vectors
    double *x, *zz, *rc, *d2, *y, *b, *w, *dy, *r64, *u, *t64;
};

__device__ __forceinline__ char* ws_ptr(const Layout& L, int a, char* smem, char* gws) {
    uint32_t o = L.off[a];
    return (o & kGlobalBit) ? gws + (o & ~kGlobalBit) : smem + o;
}

template <typename T>
__device__ inline WS<T> make_ws(const Layout& L, char* smem, char* gws, int n, int m, int q2) {
    WS<T> w;
#define P_(Ty, name, id) w.name = reinterpret_cast<Ty*>(ws_ptr(L, id, smem, gws))
    P_(uint16_t, rowent, S_ROWENT); P_(uint16_t, colent, S_COLENT);
    P_(uint16_t, rowchk, S_ROWCHK); P_(uint16_t, chkrow, S_CHKROW);
    P_(uint16_t, pivcol, S_PIVCOL); P_(uint16_t, pivrow, S_PIVROW);
    P_(uint8_t, psgn, S_PSGN);
    P_(uint16_t, lb, S_LB); P_(uint16_t, lf, S_LF);
    P_(uint32_t, lbptr, S_LBPTR); P_(uint32_t, lfptr, S_LFPTR); P_(uint32_t, cur, S_CUR);
    P_(uint16_t, lbrows, S_LBROWS); P_(uint16_t, lfrows, S_LFROWS); P_(uint16_t, selrow, S_SELROW);
    P_(uint8_t, deg, S_DEG);
    P_(uint32_t, bitmap, S_BITMAP); P_(uint8_t, flags, S_FLAGS); P_(uint32_t, mask, S_MASK);
    P_(uint32_t, flip, S_FLIP);
    T* v = reinterpret_cast<T*>(ws_ptr(L, S_VEC, smem, gws));
    w.skey = reinterpret_cast<unsigned long long*>(v);
    w.rank = reinterpret_cast<uint16_t*>(w.skey + q2);
    w.sorted = w.rank + (n + m);
    w.xs = v; v += m; w.r = v; v += m; w.z = v; v += m; w.h = v; v += m; w.l = v; v += m;
    w.t = v; v += n; w.d2t = v; v += n + m; w.invd2p = v;
    P_(double, x, G_X); P_(double, zz, G_Z); P_(double, rc, G_RC); P_(double, d2, G_D2);
    P_(double, y, G_Y); P_(double, b, G_B); P_(double, w, G_W); P_(double, dy, G_DY);
    P_(double, r64, G_R64); P_(double, u, G_U); P_(double, t64, G_T64);
    P_(uint8_t, basic, G_BASIC);
#undef P_
    return w;
}

// ---------------------------------------------------------------------------
// Block helpers
// ---------------------------------------------------------------------------
struct Blk {
    int tid, nt, lane, warp, nwarps;
    double* red;   // shared [2][64]
    int phase;
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
struct Frame {
    int p;          // LP rows
    int q;          // n + p
    double normb, normc;
};

// u^0 = bitwise hard decision (Eq. 8); empty cut set.
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
    __syncthreads();
}

// ---------------------------------------------------------------------------
// a1: cut search — Algorithm 2 per check inside the loop of Algorithm 3.
// One warp per check, lanes = neighbours (d_j <= 32).
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline int cut_search(Blk& B, const CodeView& C, WS<T>& W, const DevParams& P) {
    int added = 0;
    for (int j = B.warp; j < C.m; j += B.nwarps) {
        uint8_t f = W.flags[j];
        if ((f & kInLP) && (f & kActive)) continue;   // j has an active inequality
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
            if (B.lane == 0) { W.mask[j] = V; W.flags[j] = kInLP; }
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
// a2: augmented LP (Eq. 16) from the cut set. Coefficients are +-1:
// a_{r,i} = s_i (unflipped) or -s_i (flipped), s_i = +1 iff i in V, and
// b_r = |V| - 1 - sum_{flipped i in N(j)} s_i. The LP's pattern is packed
// per CSR edge (rowent: bit | sign) and per CSC entry (colent: LP row |
// sign, or kNone when the check is not in the LP).
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline void lp_build(Blk& B, const CodeView& C, WS<T>& W, Frame& F, int* shscan) {
    int per = (C.m + B.nt - 1) / B.nt;
    int j0 = B.tid * per, j1 = min(C.m, j0 + per);
    int cnt = 0;
    for (int j = j0; j < j1; ++j) cnt += (W.flags[j] & kInLP) ? 1 : 0;
    int total;
    int pos = bscan_excl(B, cnt, &total, shscan);
    for (int j = j0; j < j1; ++j) {
        if (W.flags[j] & kInLP) { W.rowchk[pos] = (uint16_t)j; W.chkrow[j] = (uint16_t)pos; ++pos; }
        else W.chkrow[j] = kNone;
    }
    F.p = total;
    F.q = C.n + total;
    for (int e = B.tid; e < C.E; e += B.nt) {
        int j = C.e_chk[e];
        int i = C.h_col[e];
        bool inV = (W.mask[j] >> (e - C.h_ptr[j])) & 1u;
        bool neg = inV == flipped(W.flip, i);
        W.rowent[e] = (uint16_t)(i | (neg ? kNeg : 0));
    }
    __syncthreads();
    for (int k = B.tid; k < C.E; k += B.nt) {
        uint16_t r = W.chkrow[C.v_chk[k]];
        W.colent[k] = (r == kNone) ? kNone : (uint16_t)(r | (W.rowent[C.v_eidx[k]] & kNeg));
    }
    double nb2 = 0.0;
    for (int r = B.tid; r < F.p; r += B.nt) {
        int j = W.rowchk[r];
        uint32_t V = W.mask[j];
        double shift = 0.0;
        for (int e = C.h_ptr[j]; e < C.h_ptr[j + 1]; ++e)
            if (flipped(W.flip, C.h_col[e])) shift += ((V >> (e - C.h_ptr[j])) & 1u) ? 1.0 : -1.0;
        double bv = (double)__popc(V) - 1.0 - shift;
        W.b[r] = bv;
        nb2 += bv * bv;
    }
    F.normb = sqrt(bsum(B, nb2));   // (barrier inside)
}

// (A' v)_i for a standard column i (its LP rows, through colent).
template <typename V, typename T>
__device__ __forceinline__ V colA_T(const CodeView& C, const WS<T>& W, int i, const V* v) {
    V acc = V(0);
    const int k1 = C.v_ptr[i + 1];
    for (int k = C.v_ptr[i]; k < k1; ++k) {
        uint16_t ent = W.colent[k];
        if (ent != kNone) acc += signed_val<V>(ent, v[ent & kIdx]);
    }
    return acc;
}
// (A v)_r over the standard part of LP row r (slack added by the caller).
template <typename V, typename T>
__device__ __forceinline__ V rowA(const CodeView& C, const WS<T>& W, int r, const V* vq) {
    int j = W.rowchk[r];
    V acc = V(0);
    const int e1 = C.h_ptr[j + 1];
    for (int e = C.h_ptr[j]; e < e1; ++e) {
        uint16_t ent = W.rowent[e];
        acc += signed_val<V>(ent, vq[ent & kIdx]);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// a4: column-wise greedy MTS (Algorithm 7) with weights wt[0..q).
// Columns are ranked once by (weight desc, index asc) with a bitonic sort on
// the weights rounded to FP32; DEG1 is a bitmap over ranks, so "maximum-
// weight degree-1 column" is the first set bit. Warp 0 runs the p greedy
// steps: lanes scan the bitmap and update the columns of the removed row.
// The forward-solve level of each row is fixed when its pivot is chosen and
// the back-substitution levels follow in reverse selection order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t desc_key32(float v) {
    uint32_t b = __float_as_uint(v);
    uint32_t asc = (b >> 31) ? ~b : (b | 0x80000000u);
    return ~asc;
}

__device__ inline void bitonic_sort(Blk& B, unsigned long long* key, int n2) {
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = B.tid; t < (n2 >> 1); t += B.nt) {
                int i = 2 * t - (t & (j - 1));
                int l = i + j;
                bool up = (i & k) == 0;
                unsigned long long ki = key[i], kl = key[l];
                if ((ki > kl) == up) { key[i] = kl; key[l] = ki; }
            }
            __syncthreads();
        }
    }
}

struct Levels { int nb, nf; };

template <typename T>
__device__ inline Levels mts_select(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                    const double* wt, int q2) {
    const int n = C.n, p = F.p, q = F.q;
    for (int i = B.tid; i < q; i += B.nt) {
        int dg = 1;
        if (i < n) {
            dg = 0;
            for (int k = C.v_ptr[i]; k < C.v_ptr[i + 1]; ++k) dg += (W.colent[k] != kNone);
        }
        W.deg[i] = (uint8_t)dg;
        W.pivrow[i] = kNone;
    }
    for (int k = B.tid; k < q2; k += B.nt)
        W.skey[k] = (k < q) ? (((unsigned long long)desc_key32((float)wt[k]) << 32) | (unsigned)k)
                            : ~0ull;
    for (int r = B.tid; r < p; r += B.nt) { W.pivcol[r] = kNone; W.lb[r] = 1; W.lf[r] = 1; }
    __syncthreads();
    bitonic_sort(B, W.skey, q2);
    const int nw = (q + 31) / 32;
    for (int k = B.tid; k < nw; k += B.nt) W.bitmap[k] = 0;
    for (int k = B.tid; k < q; k += B.nt) {
        int i = (int)(W.skey[k] & 0xffffffffu);
        W.rank[i] = (uint16_t)k;
        W.sorted[k] = (uint16_t)i;
    }
    __syncthreads();
    for (int i = B.tid; i < q; i += B.nt)
        if (W.deg[i] == 1) atomicOr(&W.bitmap[W.rank[i] >> 5], 1u << (W.rank[i] & 31));
    __syncthreads();

    if (B.warp == 0) {
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
                int beg = C.v_ptr[i], d = C.v_ptr[i + 1] - beg;
                unsigned cand = 0xffffffffu;
                int lv = 0;
                for (int t = lane; t < d; t += 32) {
                    uint16_t ent = W.colent[beg + t];
                    if (ent != kNone) {
                        int r = ent & kIdx;
                        if (W.pivcol[r] == kNone) cand = min(cand, (unsigned)r);
                        else lv = max(lv, (int)W.lf[r]);
                    }
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
            int j = W.rowchk[jr];
            int beg = C.h_ptr[j], d = C.h_ptr[j + 1] - beg;
            for (int t = lane; t <= d; t += 32) {
                int i2 = (t < d) ? (W.rowent[beg + t] & kIdx) : n + jr;
                if (W.pivrow[i2] != kNone) continue;   // taken (includes i)
                int nd = (int)W.deg[i2] - 1;
                W.deg[i2] = (uint8_t)nd;
                int rk = W.rank[i2];
                if (nd == 1) atomicOr(&W.bitmap[rk >> 5], 1u << (rk & 31));
                else if (nd == 0) atomicAnd(&W.bitmap[rk >> 5], ~(1u << (rk & 31)));
            }
            __syncwarp();
        }
        // back-substitution levels, in reverse selection order
        for (int k = p - 1; k >= 0; --k) {
            int r = W.selrow[k];
            int i0 = W.pivcol[r];
            int j = W.rowchk[r];
            int beg = C.h_ptr[j], d = C.h_ptr[j + 1] - beg;
            int lv = 0;
            for (int t = lane; t < d; t += 32) {
                int i2 = W.rowent[beg + t] & kIdx;
                if (i2 != i0) {
                    uint16_t pr = W.pivrow[i2];
                    if (pr != kNone) lv = max(lv, (int)W.lb[pr]);
                }
            }
            lv = (int)__reduce_max_sync(kFull, (unsigned)lv) + 1;
            if (lane == 0) W.lb[r] = (uint16_t)lv;
            __syncwarp();
        }
    }
    __syncthreads();
    // level buckets (counting sort) for both solves; pivot signs
    int mb = 0, mf = 0;
    for (int r = B.tid; r < p; r += B.nt) {
        mb = max(mb, (int)W.lb[r]);
        mf = max(mf, (int)W.lf[r]);
        int i0 = W.pivcol[r];
        uint8_t s = 0;
        if (i0 < n) {
            for (int k = C.v_ptr[i0]; k < C.v_ptr[i0 + 1]; ++k) {
                uint16_t ent = W.colent[k];
                if (ent != kNone && (ent & kIdx) == r) s = (ent & kNeg) ? 1 : 0;
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
    return L;
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

// ---------------------------------------------------------------------------
// a5: M-solve (Section V): A_M f1 = r by back substitution over the upper-
// triangular order of Algorithm 7, f2 = f1 / d_M^2, then A_M' z = f2 by
// forward substitution. Both run level by level. out[r] first holds the
// value of r's pivot column in f1, then z_r. If alpha != 0, the PCG update
// r -= alpha l, xs += alpha h of each row is fused into its back-
// substitution step.
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline void msolve(Blk& B, const CodeView& C, WS<T>& W, const Levels& L,
                              T* rvec, T* out, T alpha) {
    for (int lev = 1; lev <= L.nb; ++lev) {
        const int i1 = W.lbptr[lev + 1];
        for (int idx = W.lbptr[lev] + B.tid; idx < i1; idx += B.nt) {
            int r = W.lbrows[idx];
            T rv = rvec[r];
            if (alpha != T(0)) {
                rv -= alpha * W.l[r];
                rvec[r] = rv;
                W.xs[r] += alpha * W.h[r];
            }
            int i0 = W.pivcol[r];
            int j = W.rowchk[r];
            T acc = rv;
            const int e1 = C.h_ptr[j + 1];
            for (int e = C.h_ptr[j]; e < e1; ++e) {
                uint16_t ent = W.rowent[e];
                int i2 = ent & kIdx;
                if (i2 == i0) continue;
                uint16_t pr = W.pivrow[i2];
                if (pr != kNone) acc -= signed_val<T>(ent, out[pr]);
            }
            out[r] = W.psgn[r] ? -acc : acc;
        }
        __syncthreads();
    }
    const int n = C.n;
    for (int lev = 1; lev <= L.nf; ++lev) {
        const int i1 = W.lfptr[lev + 1];
        for (int idx = W.lfptr[lev] + B.tid; idx < i1; idx += B.nt) {
            int r = W.lfrows[idx];
            int i0 = W.pivcol[r];
            T acc = out[r] * W.invd2p[r];
            if (i0 < n) {
                const int k1 = C.v_ptr[i0 + 1];
                for (int k = C.v_ptr[i0]; k < k1; ++k) {
                    uint16_t ent = W.colent[k];
                    if (ent == kNone) continue;
                    int r2 = ent & kIdx;
                    if (r2 != r) acc -= signed_val<T>(ent, out[r2]);
                }
            }
            out[r] = W.psgn[r] ? -acc : acc;
        }
        __syncthreads();
    }
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

// PCG (Algorithm 4) in type T on Q xs = r (right side in W.r, overwritten by
// the residual), x0 = 0, stopping when ||r||_2 < tol ||rhs||_2 or after
// max_it iterations. Dot products accumulate in FP64.
template <typename T>
__device__ inline int pcg(Blk& B, const CodeView& C, WS<T>& W, const Frame& F, const Levels& L,
                          double tol, int max_it, double* relres) {
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
        T alpha = (T)(zr / hl);
        msolve<T>(B, C, W, L, W.r, W.z, alpha);   // fused r -= a l, xs += a h
        double zr_l = 0.0, rr_l = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            zr_l += (double)W.z[r] * (double)W.r[r];
            rr_l += (double)W.r[r] * (double)W.r[r];
        }
        s = bsum2(B, zr_l, rr_l);
        T nu = (T)(s.x / zr);
        zr = s.x;
        rr = s.y;
        for (int r = B.tid; r < p; r += B.nt) W.h[r] = W.z[r] + nu * W.h[r];
        __syncthreads();
        ++it;
    }
    *relres = sqrt(rr) / rn0;
    return it;
}

// Newton solve (A D^2 A') dy = w with iterative refinement: each round
// solves Q d = r64 / ||r64|| by PCG in type T, adds ||r64|| d to the FP64
// solution dy and recomputes the FP64 residual r64 = w - Q dy with FP64 D^2.
// Stops at ||r64|| < tol ||w||, when a round no longer halves ||r64||, or
// when the PCG iteration budget is spent. In FP64 mode one round normally
// suffices.
struct NewtonOut { int iters; double relres; };

template <typename T>
__device__ inline NewtonOut newton_solve(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                         const Levels& L, const DevParams& P, double tol,
                                         int max_it) {
    const int n = C.n, p = F.p;
    double ww = 0.0;
    for (int r = B.tid; r < p; r += B.nt) { W.dy[r] = 0.0; W.r64[r] = W.w[r]; ww += W.w[r] * W.w[r]; }
    const double wn = sqrt(bsum(B, ww));
    NewtonOut o{0, 0.0};
    if (wn == 0.0) return o;
    double rn = wn;
    for (int round = 0; round < 8; ++round) {
        if (rn < tol * wn || o.iters >= max_it) break;
        const double inv = 1.0 / rn;
        for (int r = B.tid; r < p; r += B.nt) W.r[r] = (T)(W.r64[r] * inv);
        __syncthreads();
        double target = tol * wn / rn;
        if (sizeof(T) < 8) target = fmax(target, P.tol_inner);
        double rel;
        o.iters += pcg<T>(B, C, W, F, L, target, max_it - o.iters, &rel);
        for (int r = B.tid; r < p; r += B.nt) W.dy[r] += rn * (double)W.xs[r];
        __syncthreads();
        // r64 = w - A D^2 A' dy in FP64
        for (int i = B.tid; i < n; i += B.nt) W.t64[i] = W.d2[i] * colA_T<double>(C, W, i, W.dy);
        __syncthreads();
        double rr = 0.0;
        for (int r = B.tid; r < p; r += B.nt) {
            double v = W.w[r] - (rowA<double>(C, W, r, W.t64) + W.d2[n + r] * W.dy[r]);
            W.r64[r] = v;
            rr += v * v;
        }
        double rn_new = sqrt(bsum(B, rr));
        bool stalled = !(rn_new < 0.5 * rn);
        rn = rn_new;
        if (stalled) break;
    }
    o.relres = rn / wn;
    return o;
}

// ---------------------------------------------------------------------------
// a3 + a6: infeasible primal-dual path-following method (Section IV-B)
// ---------------------------------------------------------------------------
struct IpmOut { int iters, pcg_iters, converged, max_levels; };

__device__ __forceinline__ double cost_of(const double* gamma, int n, int i) {
    return i < n ? fabs(gamma[i]) : 0.0;
}

// trace (optional): per iteration 8 doubles {gap, feas_p, feas_d, PCG
// iterations, Newton relative residual, beta_P, beta_D, levels}
template <typename T>
__device__ inline IpmOut ipm_solve(Blk& B, const CodeView& C, WS<T>& W, Frame& F,
                                   const DevParams& P, const double* gamma, int q2,
                                   double* trace = nullptr, int max_trace = 0) {
    const int n = C.n, p = F.p, q = F.q;
    IpmOut o{0, 0, 0, 0};
    // cold start x = e, y = 0, z = c + e
    double nc2 = 0.0;
    for (int i = B.tid; i < q; i += B.nt) {
        double c = cost_of(gamma, n, i);
        W.x[i] = 1.0;
        W.zz[i] = c + 1.0;
        nc2 += c * c;
    }
    for (int r = B.tid; r < p; r += B.nt) W.y[r] = 0.0;
    F.normc = sqrt(bsum(B, nc2));   // (barrier inside)
    for (int it = 0;; ++it) {
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
        Levels L = mts_select<T>(B, C, W, F, W.d2, q2);
        o.max_levels = max(o.max_levels, max(L.nb, L.nf));
        for (int i = B.tid; i < q; i += B.nt) W.d2t[i] = (T)W.d2[i];
        for (int r = B.tid; r < p; r += B.nt) {
            int pc = W.pivcol[r];
            W.invd2p[r] = pc < q ? (T)(1.0 / W.d2[pc]) : T(0);
        }
        __syncthreads();
        const double tol = fmax(P.tol_pcg, fmin(1e-3, P.pcg_gap_factor * g_rel));
        NewtonOut no = newton_solve<T>(B, C, W, F, L, P, tol, P.max_pcg);
        o.pcg_iters += no.iters;
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
            double* tr = trace + 8 * it;
            tr[0] = g_rel; tr[1] = fp; tr[2] = fd; tr[3] = no.iters; tr[4] = no.relres;
            tr[5] = bp; tr[6] = bd; tr[7] = max(L.nb, L.nf);
        }
        for (int i = B.tid; i < q; i += B.nt) {
            W.x[i] += bp * W.rc[i];
            W.zz[i] += bd * W.d2[i];
        }
        for (int r = B.tid; r < p; r += B.nt) W.y[r] += bd * W.dy[r];
        __syncthreads();
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
__device__ inline int vertex_recover(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
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
        int j = W.rowchk[r];
        double acc = 0.0;
        for (int e = C.h_ptr[j]; e < C.h_ptr[j + 1]; ++e) {
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

// u from x (undo the flip of Eq. 16) and the active flags of the LP rows.
template <typename T>
__device__ inline void lp_finish(Blk& B, const CodeView& C, WS<T>& W, const Frame& F,
                                 const DevParams& P) {
    for (int i = B.tid; i < C.n; i += B.nt) W.u[i] = flipped(W.flip, i) ? 1.0 - W.x[i] : W.x[i];
    for (int r = B.tid; r < F.p; r += B.nt) {
        int j = W.rowchk[r];
        W.flags[j] = kInLP | ((W.x[C.n + r] <= P.tau_act) ? kActive : 0);
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

template <typename T>
__device__ inline void decode_frame(Blk& B, const CodeView& C, WS<T>& W, const DevParams& P,
                                    const double* gamma, FrameOut out, int q2, int* shscan) {
    int bad = 0;
    for (int i = B.tid; i < C.n; i += B.nt) bad |= !isfinite(gamma[i]);
    bad = __syncthreads_or(bad);
    Frame F{0, C.n, 0.0, 0.0};
    lpdec_stats st{};
    if (bad) {
        st.status = LPDEC_ERR_INVALID_ARG;
        for (int i = B.tid; i < C.n; i += B.nt) { out.u[i] = NAN; out.hard[i] = 0; }
        if (out.mask) for (int j = B.tid; j < C.m; j += B.nt) out.mask[j] = 0;
        if (B.tid == 0) { *out.cert = 0; if (out.stats) *out.stats = st; }
        __syncthreads();
        return;
    }
    frame_init<T>(B, C, W, gamma);
    int status = LPDEC_OK;
    for (;;) {
        if (P.variant == LPDEC_MALP_B) drop_inactive<T>(B, C, W);
        int added = cut_search<T>(B, C, W, P);
        if (!added) break;
        if (st.alp_iters >= P.max_alp) { status = LPDEC_ERR_NOT_CONVERGED; break; }
        lp_build<T>(B, C, W, F, shscan);
        IpmOut io = ipm_solve<T>(B, C, W, F, P, gamma, q2);
        st.alp_iters++;
        st.ipm_iters_total += io.iters;
        st.pcg_iters_total += io.pcg_iters;
        st.max_levels = max(st.max_levels, io.max_levels);
        st.vertex_failures += vertex_recover<T>(B, C, W, F, gamma);
        lp_finish<T>(B, C, W, F, P);
        st.lp_rows_final = F.p;
        if (!io.converged) { status = LPDEC_ERR_NOT_CONVERGED; break; }
    }
    // a7: outputs. cert = integral; hard_i = [u_i > 1/2], the channel's
    // decision where u_i is within tau_int of 1/2.
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
        if (out.stats) *out.stats = st;
    }
    __syncthreads();
}

}  // namespace lpdec
