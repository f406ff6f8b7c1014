/*
 * lpdec.h — C ABI of the GB300 (sm_103a) adaptive LP decoder.
 *
 * The library decodes binary linear codes by linear programming as in
 * Taghavi, Shokrollahi, Siegel, "Efficient Implementation of Linear
 * Programming Decoding":
 *   - the code is given by its parity-check matrix H (m x n, Section II-A),
 *     passed in CSR form;
 *   - each frame is given by its LLR costs gamma (Eq. 4);
 *   - the decoder runs MALP-A (Algorithm 3) or MALP-B (Section III-A), with
 *     the O(d_j) cut search of Algorithm 2;
 *   - every LP is solved by the infeasible primal-dual path-following
 *     method of Section IV-B, whose normal equations (Eq. 24) are solved by
 *     PCG (Algorithm 4) with the column-wise maximum-weight triangular-set
 *     preconditioner (Section V, Algorithm 7);
 *   - the result is the LP solution u, its hard decision and the ML
 *     certificate flag (Section II-B: an integral u is the ML codeword).
 *
 * All work runs in CUDA kernels on one GPU. There is no CPU fallback: every
 * entry point that computes returns LPDEC_ERR_CUDA or LPDEC_ERR_NO_DEVICE
 * when no usable device is present.
 *
 * Conventions
 *   - Return value: 0 (LPDEC_OK) or a negative LPDEC_ERR_* code. No C++
 *     exception crosses this boundary.
 *   - "host" pointers are ordinary CPU memory owned by the caller; the call
 *     copies inputs before it returns and has written outputs when it
 *     returns. "device" pointers are CUDA global memory of the context's
 *     device, owned by the caller; *_device entry points are asynchronous
 *     on the given stream (a cudaStream_t passed as void*, NULL = legacy
 *     default stream) and the caller synchronises.
 *   - A context's device scratch (per-CTA workspaces, the frame queue
 *     counter, the frame-order keys) serves one batch at a time: calls on
 *     one context must run in order on the GPU (one stream, or synchronised
 *     between streams); decode concurrently with one context per stream.
 *   - Frame-major layout: array "[nframes x n]" holds frame f at offset f*n.
 *   - Cut masks: for check j, bit e of mask[j] is set iff the e-th
 *     neighbour of j (in the CSR column order of row j) belongs to the odd
 *     set V of j's parity inequality (Eq. 5). mask[j] = 0 when j has no
 *     inequality in the final LP. Check degrees must be <= 32.
 */
#ifndef LPDEC_H
#define LPDEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (return values and lpdec_stats.status). */
#define LPDEC_OK                 0
#define LPDEC_ERR_INVALID_ARG   -1  /* bad size, CSR, degree > 32, non-finite gamma */
#define LPDEC_ERR_OUT_OF_BUDGET -2  /* request exceeds the context's HBM budget; per frame:
                                       the LP outgrew its row capacity (lp_rows_cap) */
#define LPDEC_ERR_NOT_CONVERGED -3  /* an iteration cap was reached (per frame) */
#define LPDEC_ERR_TIMEOUT       -4  /* a bounded wait expired */
#define LPDEC_ERR_PENDING       -5  /* result not ready yet */
#define LPDEC_ERR_CUDA          -6  /* a CUDA runtime call failed */
#define LPDEC_ERR_NO_DEVICE     -7  /* no CUDA device / unsupported architecture */
#define LPDEC_ERR_CANCELLED     -8  /* per frame (serving): cancelled while it ran */

/* Adaptive-LP variants (Section III-A, Algorithm 1). */
#define LPDEC_MALP_A 0
#define LPDEC_MALP_B 1
#define LPDEC_ALP    2   /* Algorithm 1: inequalities are only added; every check
                            is searched in every round */

/* Preconditioner of the Newton systems (Section V): the maximum-weight
 * triangular set found by */
#define LPDEC_MTS_COLUMN      0   /* the column-wise greedy search (Algorithm 7) */
#define LPDEC_MTS_INCREMENTAL 1   /* the incremental greedy search (Algorithm 6, with the
                                     triangulation step of Algorithm 5) */
#define LPDEC_MTS_ROWWISE     2   /* the row-wise greedy search with diagonal expansion
                                     (Algorithm 8) */
#define LPDEC_MTS_ADAPTIVE    3   /* column-wise; an LP switches to the incremental search
                                     for its remaining Newton systems once one needed more
                                     than precond_switch PCG iterations */
#define LPDEC_MTS_ROWWISE_TRI 4   /* the row-wise greedy search with the triangular
                                     expansion of Section V-A: the search is run again
                                     on the columns free of the rows peeled so far,
                                     until every row is peeled */

/* Arithmetic of the PCG solve (the IPM state is always FP64). */
#define LPDEC_FP64  0   /* FP64 PCG */
#define LPDEC_MIXED 1   /* FP32 PCG inner solves refined against FP64 residuals */
#define LPDEC_M32   2   /* FP64 PCG whose preconditioner solve (the two triangular
                           sweeps of Section V) runs in FP32; flexible direction
                           update (Polak-Ribiere) */

/*
 * Tolerances and rules the paper leaves open (its Section VII lists the
 * stopping criteria and step sizes as future work). Defaults from
 * lpdec_default_params():
 *   sigma    = 0.1    centering: mu = sigma * x'z / q (Eq. 28 with sigma)
 *   eta      = 0.99   step length = min(1, eta * step to the boundary)
 *   tol_gap  = 1e-8   stop when x'z / (1 + |c'x|) < tol_gap
 *   tol_feas = 1e-8   ... and ||r_b||/(1+||b||), ||r_c||/(1+||c||) < tol_feas
 *   tol_pcg  = 1e-10  floor of the Newton-solve tolerance ||r||_2 / ||w||_2
 *   pcg_gap_factor = 0.01  inexact Newton: tolerance max(tol_pcg, min(1e-3, 0.01 * gap))
 *   tol_inner = 1e-5  relative tolerance of each FP32 PCG round (LPDEC_MIXED)
 *   tol_feas_loose = 1e-6  the IPM also stops when the gap is below tol_gap and
 *                     both infeasibilities are below this (limited accuracy of
 *                     the Newton solves near the optimum)
 *   tol_cert = 1e-3   below this gap, each interior-point iteration tries to
 *                     certify the basis of its MTS selection as optimal
 *                     (x_M = A_M^-1 b >= 0, reduced costs >= 0, complementary;
 *                     two triangular solves) and stops if it succeeds
 *   tau_act  = 1e-9   an inequality is active iff its slack <= tau_act
 *   tau_cut  = 1e-9   a check is violated iff Eq. 6's left side < 1 - tau_cut
 *   tau_int  = 1e-9   u is integral iff max |u_i - round(u_i)| <= tau_int
 *   tau_inc  = 1e-9   Theorem 2(b): with unique LP optima the MALP cost
 *                     gamma'u rises strictly from LP to LP. A MALP frame whose
 *                     new LP cost is not above the previous one by more than
 *                     tau_inc * (1 + |previous|) has an optimum that is not
 *                     unique, where MALP can cycle between cut sets short of
 *                     the LP decoding optimum; it continues as ALP
 *                     (Algorithm 1) from its cut set, which only adds
 *                     inequalities and reaches the optimum (Theorem 2(c);
 *                     stats.alp_switch records when).
 *   max_alp = 200, max_ipm = 60, max_pcg = 1000 iteration caps (max_pcg per
 *                     Newton solve, over all refinement rounds; an LP whose
 *                     interior-point run converges needs at most ~40
 *                     iterations on the workloads measured). A Newton solve
 *                     whose PCG misses its tolerance within max_pcg (CG needs
 *                     at most p steps in exact arithmetic, so it has stalled)
 *                     is redone by a dense FP64 Cholesky factorization of
 *                     A D^2 A' (LPs of up to 2048 rows), and so are the
 *                     remaining Newton solves of that LP
 *   dense_switch = 64 a Newton solve whose PCG converges only after more
 *                     than 64 max(1, (p/512)^2) iterations also sends the
 *                     rest of its LP to the dense solve (cheaper there)
 *   order_frames = 1  frames of a one-code batch with more frames than CTAs
 *                     are handed out hardest first (results unchanged)
 *   variant = LPDEC_MALP_A, precision = LPDEC_FP64
 *   precond = LPDEC_MTS_COLUMN, precond_switch = 150, warm_start = 0,
 *   mts_reuse = 0 (the paper's future work, Sections V and VII: the
 *   previous iterate and triangular set reused; results are the same
 *   certified vertices either way)
 *   lp_rows_cap = 0   rows one frame's LP may hold (0 = 2m). The main
 *                     workspace holds min(m, lp_rows_cap) rows, enough for
 *                     MALP (one inequality per check); a frame whose cut list
 *                     grows past it (ALP, or MALP continued as ALP) moves to
 *                     a wide workspace in global scratch; a frame whose cut
 *                     list outgrows lp_rows_cap ends with
 *                     LPDEC_ERR_OUT_OF_BUDGET
 * The decisions are taken on the LP's optimal vertex, recovered from the
 * final interior-point iterate through its strictly complementary
 * partition (basic iff x_i > z_i, Section VI-A) and certified optimal by a
 * primal-dual feasible, complementary pair. An iterate whose partition does
 * not certify (it has not separated yet) is refined by solving the LP again
 * at a 100x, then 1000x tighter gap with twice max_ipm; an LP that still
 * cannot be certified keeps the partition's vertex and counts in
 * stats.vertex_failures.
 */
typedef struct lpdec_params {
    double sigma, eta, tol_gap, tol_feas, tol_pcg, tau_act, tau_cut, tau_int;
    double pcg_gap_factor;  /* Newton solve tolerance = max(tol_pcg, min(1e-3, f * gap)) */
    double tol_inner;       /* relative tolerance of one FP32 PCG round (LPDEC_MIXED) */
    double tol_feas_loose;  /* infeasibility accepted once the gap is below tol_gap */
    double tol_cert;        /* gap below which the optimality certificate is tried */
    double tau_inc;         /* least relative cost rise from one LP to the next */
    int32_t max_alp, max_ipm, max_pcg, variant, precision;
    int32_t threads_per_block;  /* 0 = library choice */
    int32_t smem_budget;        /* bytes of shared memory per CTA, 0 = library choice */
    int32_t lp_rows_cap;        /* LP row capacity per frame, 0 = library choice */
    int32_t precond;            /* LPDEC_MTS_* */
    int32_t precond_switch;     /* PCG iterations of one Newton solve after which
                                   LPDEC_MTS_ADAPTIVE switches the LP to Algorithm 6 */
    int32_t warm_start;         /* 1: each LP of a MALP frame after the first starts the
                                   interior-point method from the previous LP's final
                                   iterate (x, z floored at 0.01; rows kept from the
                                   previous LP keep their slack and dual, new rows start
                                   cold); 0: cold start (R4) */
    int32_t mts_reuse;          /* 1: an interior-point iteration keeps the previous
                                   triangular set while the last PCG took <= 20
                                   iterations and the partition x_i > z_i kept its size
                                   (the values of M are always current) */
    int32_t lane_policy;        /* lanes per row in the single-warp levels of the
                                   triangular solves: 0 = by the level's width (8 lanes
                                   for up to 4 rows, 4 up to 8, 2 up to 16, else 1), or a
                                   fixed 1, 2, 4 or 8 (see lpdec_autotune) */
    int32_t order_frames;       /* order in which the CTAs of a one-code batch take its
                                   frames: 0 = as given; 1 (default) = when more frames
                                   than CTAs, those expected to need the most LPs first
                                   (largest sum of -gamma_i over gamma_i < 0), so the
                                   slow ones do not start last; 2 = always. Results do
                                   not depend on the order. */
    int32_t dense_switch;       /* a Newton solve whose PCG converges after more than
                                   dense_switch max(1, (p/512)^2) iterations (p the
                                   LP's rows) sends the rest of its LP's Newton solves
                                   to the dense Cholesky fallback (when the LP fits
                                   it); 0 = only after PCG stalls. A dense solve costs
                                   p^3/6 FMAs, a PCG iteration about p dependent steps;
                                   default 64 (on GB300 a dense solve at 512 rows costs
                                   about as much as that many PCG iterations) */
    int32_t reserved;
} lpdec_params;

/* Per-frame results besides u / hard / cert. */
typedef struct lpdec_stats {
    int32_t status;           /* LPDEC_OK, or LPDEC_ERR_NOT_CONVERGED / OUT_OF_BUDGET / INVALID_ARG */
    int32_t alp_iters;        /* number of LPs solved (0 if the hard decision is a codeword) */
    int32_t ipm_iters_total;  /* interior-point iterations over all LPs */
    int32_t pcg_iters_total;  /* PCG iterations over all Newton steps */
    int32_t lp_rows_final;    /* p of the last LP (parity inequalities) */
    int32_t vertex_failures;  /* LPs whose vertex could not be certified optimal */
    int32_t max_levels;       /* deepest triangular-solve level schedule seen */
    int32_t pcg_iters_fp64;   /* PCG iterations run in FP64 (all of them in LPDEC_FP64) */
    int32_t dense_solves;     /* Newton systems solved by the dense Cholesky fallback */
    int32_t alp_switch;       /* LPs solved before a MALP frame continued as ALP (0: never) */
    int32_t lp_rows_max;      /* rows of the largest LP solved */
    int32_t ipm_iters_refine; /* of ipm_iters_total: iterations of the re-solves at a
                                 tighter gap of LPs whose vertex failed the certificate */
    double  objective;        /* gamma'u */
    double  pcg_flops;        /* algorithmic floating-point operations of the Newton
                                 solves: PCG iterations (Q h, both triangular
                                 solves, dots, updates), the FP64 residuals of
                                 refinement and any dense fallback */
    double  seconds;          /* device time from the frame's start to its end
                                 (batch entry points: its time on its CTA) */
    double  pcg_bytes;        /* algorithmic bytes of the PCG iterations of a
                                 frame streamed from memory: per iteration, both
                                 index passes and D^2 of Q h (4-byte indices),
                                 its two vectors, the two triangular solves
                                 (4 nnz(A_M) + 8p each) and five 8p vector passes */
    double  t_start, t_end;   /* device global timer (ns) at the frame's start and end */
    /* device time (s) of the frame's phases, from the global timer: */
    double  sec_mts;          /* triangular-set selections and their level schedules */
    double  sec_pcg;          /* Newton solves by PCG (with FP64 refinement) */
    double  sec_dense;        /* Newton solves that ended in the dense fallback */
    double  sec_certify;      /* vertex certificates (basis and general) and recovery */
    double  sec_refine;       /* re-solves at a tighter gap, all their phases included
                                 (so overlapping the four above) */
} lpdec_stats;

typedef struct lpdec_ctx lpdec_ctx;    /* opaque: device, streams, scratch */
typedef struct lpdec_code lpdec_code;  /* opaque: device copy of H (CSR + CSC) */

/* Fills *p with the defaults listed above. */
void lpdec_default_params(lpdec_params* p);

/* Static string for a status code. */
const char* lpdec_error_string(int32_t code);

/* Host-only (no device needed): the per-frame workspace of a code with m
 * checks, n bits and E edges (check degrees at most ceil(E/m)) in the given
 * precision mode, with the default parameters — shared memory per CTA
 * (*smem_bytes) and global scratch per concurrently decoded frame
 * (*global_bytes_per_frame, including the dense fallback's matrix when the
 * LP row capacity is <= 2048) — for a shared-memory budget per CTA
 * (smem_budget <= 0: 227 KB, the largest layout; the decoder itself
 * defaults to a third of the SM's shared memory, 75 KB on GB300). Also
 * validates the layout (every array aligned, inside its region, disjoint
 * from the others). */
int32_t lpdec_workspace_bytes(int32_t m, int32_t n, int32_t E, int32_t precision,
                              int32_t smem_budget, size_t* smem_bytes,
                              size_t* global_bytes_per_frame);

/* Creates a context on CUDA device `device`. `params` may be NULL
 * (defaults). `hbm_budget_bytes` bounds the scratch the context may hold
 * (0 = no bound). Returns LPDEC_ERR_NO_DEVICE without a usable device. */
int32_t lpdec_ctx_create(int32_t device, const lpdec_params* params,
                         size_t hbm_budget_bytes, lpdec_ctx** out);
void lpdec_ctx_destroy(lpdec_ctx* ctx);

/* Replaces the context's parameters (takes effect at the next call). */
int32_t lpdec_ctx_set_params(lpdec_ctx* ctx, const lpdec_params* params);

/* Uploads H (m x n) given in CSR form on the host: row_ptr[m+1],
 * col_idx[row_ptr[m]] with strictly increasing columns in each row.
 * Validates the CSR, that every row has 1..32 entries and that
 * m, n <= 32767 (the kernels pack indices into 15 bits). Decoding further
 * needs the arrays that always live in shared memory (about 12 bytes per
 * check plus one bit per column, see lpdec_workspace_bytes) to fit one
 * CTA's shared memory (227 KB): m up to about 18,000. Larger codes are
 * rejected by the decode calls with
 * LPDEC_ERR_INVALID_ARG. The code may be used with any context on the same
 * device. */
int32_t lpdec_code_create(lpdec_ctx* ctx, int32_t m, int32_t n,
                          const int32_t* row_ptr, const int32_t* col_idx,
                          lpdec_code** out);
void lpdec_code_destroy(lpdec_code* code);

/* Decodes one frame (host pointers). gamma[n] in; u_out[n], hard_out[n],
 * cert_out[1] out; cut_mask_out[m] and stats optional (NULL). */
int32_t lpdec_decode(lpdec_ctx* ctx, const lpdec_code* code, const double* gamma,
                     double* u_out, uint8_t* hard_out, int32_t* cert_out,
                     uint32_t* cut_mask_out, lpdec_stats* stats);

/* Decodes a batch of frames, each with its own code (the problem statement
 * of Section II-A/B per frame: H and gamma in; u, hard decision and ML
 * certificate out). Host pointers, one per frame: codes[f] (a code of any
 * context on this context's device), gammas[f][n_f] in; u_out[f][n_f],
 * hard_out[f][n_f], cert_out[nframes] out; cut_mask_out (NULL, or one
 * pointer per frame, each NULL or [m_f]) and stats[nframes] optional. All
 * frames, whatever their code lengths, share one persistent launch; the
 * call packs them, copies in and out, and returns when the outputs are
 * written. Returns LPDEC_ERR_INVALID_ARG for a NULL pointer, a non-finite
 * LLR or a code of another device; per-frame failures are in stats. */
int32_t lpdec_decode_batch(lpdec_ctx* ctx, int32_t nframes, const lpdec_code* const* codes,
                           const double* const* gammas, double* const* u_out,
                           uint8_t* const* hard_out, int32_t* cert_out,
                           uint32_t* const* cut_mask_out, lpdec_stats* stats);

/* Decodes nframes frames of one code (host pointers, frame-major):
 * gamma[nframes x n] in; u_out[nframes x n], hard_out[nframes x n],
 * cert_out[nframes] out; cut_mask_out[nframes x m] and stats[nframes]
 * optional. Copies in and out inside the call. */
int32_t lpdec_decode_frames(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                            const double* gamma, double* u_out, uint8_t* hard_out,
                            int32_t* cert_out, uint32_t* cut_mask_out, lpdec_stats* stats);

/* Same as lpdec_decode_frames with DEVICE pointers, asynchronous on
 * `stream`. d_cut_mask and d_stats may be NULL. One persistent kernel
 * decodes all frames; CTAs take frames from a queue. */
int32_t lpdec_decode_batch_device(lpdec_ctx* ctx, const lpdec_code* code,
                                  int32_t nframes, const double* d_gamma,
                                  double* d_u, uint8_t* d_hard, int32_t* d_cert,
                                  uint32_t* d_cut_mask, lpdec_stats* d_stats,
                                  void* stream);

/* Launch shape of a one-code batch under the context's parameters (host
 * query, no allocation, no launch): *grid = the CTAs (persistent, one frame
 * at a time each) that lpdec_decode_frames / lpdec_decode_batch_device use
 * for nframes frames of `code` (0 for none); *ordered (may be NULL) = 1 when
 * that batch is handed out in the hardest-first order of order_frames, which
 * adds two small kernels (keys, sort) before the decode kernel. Returns
 * LPDEC_ERR_INVALID_ARG for a NULL pointer, nframes < 0, a code of another
 * device, or a code whose workspace does not fit an SM. */
int32_t lpdec_batch_grid(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                         int32_t* grid, int32_t* ordered);

/* Device form of lpdec_decode_batch, asynchronous on `stream`: codes is a
 * HOST array of nframes code handles; the device arrays are ragged and
 * frame-major: frame f's bits start at n_0 + ... + n_{f-1} in d_gamma, d_u,
 * d_hard, its checks at m_0 + ... + m_{f-1} in d_cut_mask (optional), and
 * d_cert / d_stats (optional) hold one entry per frame. The code table and
 * frame descriptors are copied to the context's device buffer on `stream`;
 * the workspace is laid out for the largest code of the batch. */
int32_t lpdec_decode_mixed_device(lpdec_ctx* ctx, int32_t nframes, const lpdec_code* const* codes,
                                  const double* d_gamma, double* d_u, uint8_t* d_hard,
                                  int32_t* d_cert, uint32_t* d_cut_mask, lpdec_stats* d_stats,
                                  void* stream);

/* Schedule autotuner (no counterpart in the paper): decodes the host
 * sample gamma[nframes x n] once per candidate lanes-per-row schedule of the
 * triangular solves (lane_policy 0, 1, 2, 4, 8), keeps in the context the
 * one with the least total device time of the frames on their CTAs, and
 * writes it to *policy_out (optional); seconds_out[5] (optional) receives
 * each candidate's total. A schedule changes only the order in which a
 * row's dependency sum is added (rounding); the decoded results are the
 * same certified LP vertices. */
int32_t lpdec_autotune(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                       const double* gamma, int32_t* policy_out, double* seconds_out);

/* ---- Single steps of the hot path (device pointers, asynchronous) ----
 * These run the same device code as the decoder on caller-given state, one
 * frame per CTA, so each step can be checked on its own. "LP state" means
 * in_lp[nframes x m] (1 = check j has a parity inequality in the LP) and
 * mask[nframes x m]; the LP rows are the checks with in_lp = 1 in
 * increasing order, p = their count, q = n + p, columns n..n+p-1 are the
 * slacks (Eq. 16). Per-frame vectors over columns use a stride of n + m
 * (q <= n + m), over rows a stride of m. */

/* One round of the MALP-A / MALP-B cut search (the search step of
 * Algorithm 3, with Algorithm 2 per check) at u[nframes x n]. active[nframes x m] marks
 * checks whose inequality is active in the current LP. mask and in_lp are
 * updated in place; flag[nframes] = 1 if an inequality was added. */
int32_t lpdec_cut_search_device(lpdec_ctx* ctx, const lpdec_code* code,
                                int32_t nframes, const double* d_u,
                                const uint8_t* d_active, uint8_t* d_in_lp,
                                uint32_t* d_mask, int32_t* d_flag, void* stream);

/* Maximum-weight triangular set of the LP given by (gamma, in_lp, mask)
 * with column weights w[nframes x (n+m)] (the decoder uses w_i = d_i^2 =
 * x_i / z_i; ties go to the lower column index), by the context's
 * lpdec_params.precond: column-wise (Algorithm 7, also for
 * LPDEC_MTS_ADAPTIVE), incremental (Algorithm 6 with 5), row-wise with the
 * diagonal (Algorithm 8) or the triangular expansion (Section V-A). Writes
 * the selection order: col[nframes x m] (column chosen at step k) and
 * row[nframes x m] (its LP row); entries k >= p are -1. */
int32_t lpdec_mts_select_device(lpdec_ctx* ctx, const lpdec_code* code,
                                int32_t nframes, const double* d_gamma,
                                const uint8_t* d_in_lp, const uint32_t* d_mask,
                                const double* d_w, int32_t* d_col, int32_t* d_row,
                                void* stream);

/* One Newton solve (Eq. 24) as the decoder does it: PCG (Algorithm 4) with
 * the context's triangular-set preconditioner (weights d2; lpdec_params.
 * precond, column-wise for LPDEC_MTS_ADAPTIVE) in the context's precision
 * mode, and the dense fallback when PCG stalls, for (A D^2 A') dy = w of
 * the LP given by (gamma, in_lp, mask): d2[nframes x (n+m)], w[nframes x m]
 * in; dy[nframes x m] and iters[nframes] (PCG iterations) out. */
int32_t lpdec_pcg_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                         const double* d_gamma, const uint8_t* d_in_lp,
                         const uint32_t* d_mask, const double* d_d2,
                         const double* d_w, double* d_dy, int32_t* d_iters,
                         void* stream);

/* Diagnostic PCG (Algorithm 4, FP64, one run from dy = 0, no refinement)
 * for the preconditioner study of Section VI-B and the spectral diagnostics
 * of its closing remarks: the LP given by (gamma, in_lp, mask), weights and
 * D^2 = d2[nframes x (n+m)], right side w[nframes x m], preconditioned by
 * the context's triangular set (lpdec_params.precond) or, with identity != 0,
 * not at all (plain CG). Runs until ||r|| < tol ||w|| or max_hist
 * iterations; writes dy[nframes x m], iters[nframes] and, per frame and
 * iteration k < max_hist, hist[(f * max_hist + k) * 3 ...] = ||r_k|| / ||w||,
 * alpha_k, nu_k (zeros past the last iteration). The coefficients define
 * the Lanczos tridiagonal of the preconditioned operator (diagonal
 * 1/alpha_k + nu_{k-1}/alpha_{k-1}, off-diagonal sqrt(nu_k)/alpha_k), whose
 * extreme eigenvalues estimate its condition number. */
int32_t lpdec_pcg_trace_device(lpdec_ctx* ctx, const lpdec_code* code, int32_t nframes,
                               const double* d_gamma, const uint8_t* d_in_lp,
                               const uint32_t* d_mask, const double* d_d2, const double* d_w,
                               int32_t identity, double tol, int32_t max_hist, double* d_dy,
                               int32_t* d_iters, double* d_hist, void* stream);

/* Solves one LP (Section IV-B interior-point method + optimal-vertex
 * recovery) given by (gamma, in_lp, mask): x[nframes x (n+m)] out (the
 * recovered vertex, slacks at n..n+p-1), stats[nframes] out
 * (ipm_iters_total, pcg_iters_total, vertex_failures, status, objective). */
int32_t lpdec_lp_solve_device(lpdec_ctx* ctx, const lpdec_code* code,
                              int32_t nframes, const double* d_gamma,
                              const uint8_t* d_in_lp, const uint32_t* d_mask,
                              double* d_x, lpdec_stats* d_stats, void* stream);

/* Diagnostic form of lpdec_lp_solve_device (one interior-point run, without
 * the refinement of an uncertified vertex): also writes, per frame and per
 * interior-point iteration k < max_trace, 10 doubles to
 * trace[(f * max_trace + k) * 10 ...]: relative gap, relative primal and
 * dual infeasibility, PCG iterations, final PCG relative residual, beta_P,
 * beta_D, the deepest triangular-solve level schedule, and the smallest and
 * largest eigenvalue of the Lanczos tridiagonal of the Newton solve's first
 * PCG round (its first 64 CG coefficients): an estimate of the spectrum of
 * M^-1 Q, the preconditioned normal matrix (Section VI). */
int32_t lpdec_lp_solve_trace_device(lpdec_ctx* ctx, const lpdec_code* code,
                                    int32_t nframes, const double* d_gamma,
                                    const uint8_t* d_in_lp, const uint32_t* d_mask,
                                    double* d_x, lpdec_stats* d_stats,
                                    double* d_trace, int32_t max_trace, void* stream);

/* Allocation-free variant of lpdec_decode_batch_device (no counterpart in
 * the paper). It is for callers that cannot allocate device memory when they
 * decode — a host component that has already reserved all GPU memory, a
 * real-time loop that must stay out of the allocator — and it calls no
 * cudaMalloc, cudaFree or other allocating routine. Instead of the
 * context's scratch it uses one fixed device array of 32 MiB inside this
 * library (present on every GPU that loads the library, until the process
 * exits); the frames run on as many CTAs as fit in it.
 *   - code: from lpdec_code_create (created beforehand; its context picks
 *     the device). params: NULL = defaults; the context's parameters are
 *     not used.
 *   - Inputs and outputs are caller-owned device buffers, as in
 *     lpdec_decode_batch_device; asynchronous on `stream`.
 *   - Every call takes the array's device address (cudaGetSymbolAddress,
 *     which allocates nothing); the first call on a device may also load the
 *     module, so make it before any stream capture.
 *   - Every call uses the same array and leaves its contents behind; the
 *     call resets what must start at zero itself. Calls that overlap on the
 *     GPU (other streams, other threads) race on the array: serialize them.
 *   - The dense Cholesky fallback of stalled Newton solves runs as in the
 *     regular entry whenever one CTA's workspace with its matrix fits the
 *     array (n = 1008: about 3.9 MB per CTA, so 8 CTAs run at once instead
 *     of the regular entry's 456); only codes whose matrix alone outgrows the
 *     array run without it, and a frame whose PCG stalls there may end
 *     LPDEC_ERR_NOT_CONVERGED where the regular entry converges.
 *   - Returns LPDEC_ERR_OUT_OF_BUDGET when one frame's workspace exceeds the
 *     array (very long codes), LPDEC_ERR_INVALID_ARG for bad arguments. */
int32_t lpdec_decode_batch_device_noalloc(const lpdec_code* code,
                                          const lpdec_params* params, int32_t nframes,
                                          const double* d_gamma, double* d_u,
                                          uint8_t* d_hard, int32_t* d_cert,
                                          uint32_t* d_cut_mask, lpdec_stats* d_stats,
                                          void* stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching. The paper decodes one frame at a time and
 * has no counterpart; each frame is still decoded by Algorithm 3 exactly as
 * by lpdec_decode, and its result does not depend on the frames it shares
 * the GPU with.
 *
 * A server decodes frames of the codes it is created with (any lengths) as
 * they are submitted. One persistent kernel runs while frames are queued;
 * its CTAs take the next queued frame as soon as they finish one, so a frame
 * submitted while others run starts as soon as a CTA frees up, and the
 * kernel ends by itself once no frame has arrived for a short idle time
 * (the server starts it again on the next submission). Frames are admitted
 * by device-memory bytes: each frame holds a region of the server's arena
 * (its LLRs in, its results out: about 17 n + 4 m bytes) from submission
 * until its results are copied back, and a submission that does not fit is
 * refused. All waits inside the kernel are bounded.
 *
 * lpdec_server_create: codes[ncodes] (from lpdec_code_create, on `device`;
 * they must outlive the server); params as for lpdec_ctx_create (NULL =
 * defaults); hbm_budget_bytes bounds the device memory of the server, its
 * per-CTA scratch included (0: an arena for max_pending frames of the
 * largest code); max_pending (1 .. 2^20) bounds the frames queued or running.
 * Returns LPDEC_ERR_OUT_OF_BUDGET when the budget does not cover the
 * scratch plus one frame, LPDEC_ERR_NO_DEVICE without a usable GPU,
 * LPDEC_ERR_INVALID_ARG for bad arguments. */
typedef struct lpdec_server lpdec_server;
int32_t lpdec_server_create(int32_t device, const lpdec_params* params, int32_t ncodes,
                            const lpdec_code* const* codes, size_t hbm_budget_bytes,
                            int32_t max_pending, lpdec_server** out);

/* Queues one frame of `code` (one of the server's codes): gamma = n host
 * FP64 LLRs, copied to the device before return. Writes the frame's ticket
 * (0, 1, 2, ... in submission order). Returns LPDEC_ERR_OUT_OF_BUDGET when
 * the frame's region does not fit the arena or max_pending frames are
 * queued or running, LPDEC_ERR_INVALID_ARG for a non-finite LLR or a code
 * the server was not created with, or the server's sticky error after a
 * failed CUDA call. */
int32_t lpdec_submit(lpdec_server* server, const lpdec_code* code, const double* gamma,
                     uint64_t* ticket);

/* Result of one ticket, once: u (n FP64), hard (n bytes), cert, cut mask
 * (m words) and stats (any output may be NULL); then the ticket is
 * released. Returns LPDEC_ERR_PENDING while the frame is queued or running,
 * LPDEC_ERR_INVALID_ARG for a ticket never issued, already polled or
 * cancelled, or the server's sticky error. Never blocks on the GPU. */
int32_t lpdec_poll(lpdec_server* server, uint64_t ticket, double* u_out, uint8_t* hard_out,
                   int32_t* cert_out, uint32_t* cut_mask_out, lpdec_stats* stats);

/* Cancels a ticket: a frame no CTA has taken yet is skipped; a running one
 * stops at its next check, one every four interior-point iterations and
 * before each LP (milliseconds at the codes of the serving workloads), and
 * frees its CTA for the next frame. Either way its result is dropped and
 * its region and ticket are released once the CTA has let go of it (no
 * poll needed). LPDEC_ERR_INVALID_ARG for a ticket never issued, polled or
 * cancelled. */
int32_t lpdec_cancel(lpdec_server* server, uint64_t ticket);

/* Device bytes the server holds (scratch + arena), the arena's size, the
 * arena bytes held by frames, and the tickets not yet polled or released
 * (any output may be NULL). A frame of a code with n bits and m checks
 * holds 8n (LLRs) + 8n (u) + n (hard) + 4m (cut mask) + 4 (cert) bytes and
 * one lpdec_stats, each part 16-byte aligned, rounded up to 256 bytes. */
int32_t lpdec_server_stats(lpdec_server* server, size_t* hbm_bytes, size_t* arena_bytes,
                           size_t* arena_used, int32_t* outstanding);

/* Stops the kernel, drops queued frames and frees everything. */
int32_t lpdec_server_destroy(lpdec_server* server);

#ifdef __cplusplus
}
#endif

#endif /* LPDEC_H */
