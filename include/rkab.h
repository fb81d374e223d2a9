/*
 * rkab.h -- C ABI of the GB300 (sm_103a) library for Randomized Kaczmarz (RK),
 * Randomized Kaczmarz with Averaging (RKA) and the block-averaging variant
 * RKAB of Ferreira, Acebron and Monteiro, "Parallelization Strategies for the
 * Randomized Kaczmarz Algorithm on Large-Scale Dense Systems" (arXiv 2401.17474).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Device pointers are CUDA device addresses owned by the caller; the
 *    library keeps none of them beyond the lifetime documented for the plan
 *    and never calls cudaMalloc/cudaFree.  Scratch memory is a caller-provided
 *    workspace whose size is given by the matching *_workspace_bytes query.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work is enqueued asynchronously on it; host-side
 *    argument errors are returned immediately, device-side errors are written
 *    to a status word in the workspace and reported by rk_plan_status /
 *    rk_solve_status after the stream has been synchronised.
 *  - Return value: 0 (RK_OK) or a negative RK_E* code; no exception or
 *    longjmp crosses the ABI.  rk_strerror() names a code.
 *  - Matrices are row-major with leading dimension `lda` (elements); the
 *    base address and lda * element size must be multiples of 16 bytes (rows
 *    are moved by bulk asynchronous copies).  A holds m * lda elements; the
 *    columns n .. lda-1 may hold anything.
 *  - "Round" means one average: every worker applies `alpha` projections to
 *    its own copy of x, then the q copies are averaged.
 */
#ifndef RKAB_H
#define RKAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define RK_OK 0
#define RK_EINVAL (-1)          /* invalid argument (sizes, q, alpha, null pointer, non-finite A) */
#define RK_EALIGN (-2)          /* base address or lda * element size not a multiple of 16 bytes */
#define RK_ENOTCORESIDENT (-3)  /* the persistent grid does not fit co-resident on the device */
#define RK_ETIMEOUT (-4)        /* a device-side wait (grid barrier, copy) exceeded its limit */
#define RK_EDIVERGED (-5)       /* x became non-finite (e.g. relaxation beyond the stable range) */
#define RK_ECUDA (-6)           /* a CUDA runtime call failed */
#define RK_EWORKSPACE (-7)      /* workspace smaller than the size query returned */
#define RK_ESETUP (-8)          /* the plan's device-side setup failed (see rk_plan_status) */
#define RK_ETOOLARGE (-9)       /* q x n exceeds the fixed scratch of rkab_solve_noalloc */

/* Storage type of the rows the solver streams. */
typedef enum {
    RK_F32 = 0,       /* float32 */
    RK_BF16 = 1,      /* bfloat16, dequantised to float32 on load */
    RK_FP8E4M3 = 2    /* OCP FP8 e4m3 (finite-only variant) with one float32 scale per row */
} rk_dtype;

/* Opaque plan: the sampling tables of one matrix, living in a caller workspace. */
typedef struct rk_plan rk_plan;

/* Solver options.  rk_opts_default() fills the defaults given in brackets. */
typedef struct {
    float omega;           /* relaxation of Eq. (alg) (the paper's alpha_i / uniform weight
                              alpha of Eq. (rka_uni_weights)), in (0, 2q) for q workers:
                              one chain converges for (0, 2); the averaged step of RKA
                              takes weights up to alpha* of Eq. (best_alpha) < 2q
                              (rk_alpha_star)                                        [1.0] */
    int64_t check_every;   /* rounds between convergence checks; 0 = never          [1]   */
    double tol;            /* stop after the first checked round with metric < tol  [0]   */
    int criterion;         /* 0 none; 1 ||x - x_ref|| / ||x_ref|| (needs x_ref)    [0]   */
    const float *x_ref;    /* device, n floats: reference solution for criterion 1  [NULL]*/
    int64_t round0;        /* index of the first round (resume: the draws of a run
                              restarted at round k equal those of an uninterrupted
                              run from round k on)                                  [0]   */
    uint32_t stream_id;    /* Philox stream id of the draws: 0 rows of A, 1 rows of
                              A^T, 2 recovery solve, 3 + (outer << 8) refinement    [0]   */
    int same_stream;       /* nonzero: every worker draws worker 0's rows (test hook) [0] */
    int cluster_size;      /* CTAs per worker (1, 2, 4, 8, 16): a worker's row is split
                              into that many column chunks, one per CTA of a thread-
                              block cluster, reduced through distributed shared
                              memory; 0 or 1 = one CTA per worker                  [0]   */
    double timeout_s;      /* limit of every device-side wait, seconds              [10]  */
    int lookahead;         /* rows per look-ahead group (1, 2, 4; 6 with clusters): the dots of the
                              next rows and their pairwise products are reduced once
                              per group and the projections resolved by a scalar
                              recurrence (same result as one row at a time in exact
                              arithmetic); 0 = chosen by the library               [0]   */
    int sampling;          /* row selection (rk_sampling):
                              RK_SAMPLE_FULL   every worker draws from the whole law of
                                               Eq. (prob_line) (alias table)
                              RK_SAMPLE_BLOCKS the Distributed Approach of Section 3.3.1:
                                               worker g of q draws only from its block of
                                               rows [g m / q, (g+1) m / q), with probability
                                               ||A_i||^2 / (the block's sum)
                              RK_SAMPLE_CYCLIC worker g sweeps the rows in order from
                                               g m / q: row (g m / q + t) mod m (Section 2.1,
                                               the cyclic Kaczmarz method for q = 1)   [FULL] */
    const float *row_weight;  /* device, m floats or NULL: per-row weights w_i of Eq.
                              (rka_eq), multiplying omega in each projection        [NULL]*/
    const float *worker_weight; /* device, q floats or NULL: per-worker weights, the
                              Partial Matrix alpha of Section 3.3.1 (Table 1): every
                              projection of worker g is scaled by worker_weight[g],
                              multiplying omega and the row weight
                              (rk_partial_alpha_star computes them)                [NULL]*/
} rk_opts;

/* Row selection of rk_opts.sampling. */
typedef enum { RK_SAMPLE_FULL = 0, RK_SAMPLE_BLOCKS = 1, RK_SAMPLE_CYCLIC = 2 } rk_sampling;

void rk_opts_default(rk_opts *opts);

/* ------------------------------------------------------------------------ */
/* Setup: sampling law of Eq. (prob_line), P{i = l} = ||A_l||^2 / ||A||_F^2  */
/* (Section 2.2), its exclusive prefix sum and its alias table, plus the    */
/* float32 reciprocals 1/||A_i||^2 used by the projection of Eq. (alg).     */
/*                                                                          */
/* The law is encoded with exact integers (identical on every device and on */
/* the CPU whatever the summation order):                                   */
/*   e_i  exponent of max_j |a_ij| (max = f 2^e_i, f in [0.5, 1))           */
/*   R_i  = sum_j floor(a_ij^2 2^(102 - 2 e_i))                             */
/*   L    = max_i (bitlength(R_i) + 2 e_i - 102) + ceil(log2 m) - 62        */
/*   K_i  = floor(R_i 2^(2 e_i - 102 - L)),  T = sum_i K_i < 2^62           */
/*   P_i  = sum_{l < i} K_l (uint64 exclusive prefix)                       */
/* and the alias table (thr64_i, alias_i) of the law K_i / T is built by    */
/* the sweeping construction (lights and heavies in ascending index order). */
/* For RK_BF16 and RK_FP8E4M3 the law and the reciprocals are those of the  */
/* stored rows: a_ij is the float32 value of the stored element (times the  */
/* row scale for FP8, rounded to float32).                                  */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace rk_setup needs for an m-row matrix. */
size_t rk_setup_workspace_bytes(int64_t m, int64_t n);

/* Build a plan for A (device, m x n, row-major, leading dimension lda).
 *   A          device rows of type dt; must outlive the plan
 *   row_scale  device, m floats (FP8 only: a_ij = row_scale_i * e4m3_ij); NULL otherwise
 *   workspace  device, >= rk_setup_workspace_bytes(m, n) bytes, 256-byte aligned; owned by
 *              the caller, must outlive the plan and not be reused while the plan lives
 *   out        receives a host-allocated plan (release with rk_plan_destroy)
 * Limits: 1 <= m < 2^31, 1 <= n < 2^26, lda >= n.  Enqueues the build on `stream`;
 * an all-zero or non-finite A is reported by rk_plan_status (RK_ESETUP), and so is a
 * row the law can draw (K_i > 0) whose ||A_i||^2 lies outside [2^-126, 2^126): the
 * float32 projection of Eq. (alg) cannot take it (1/||A_i||^2 overflows, the products
 * <A_i, x> underflow).  Eq. (alg) is invariant under scaling a row and its b_i by the
 * same factor, so such a system is solved after scaling A and b by a power of two
 * (exact in float32), which leaves x unchanged.  Rows outside that range that the law
 * never draws (their weight truncates to K_i = 0) keep the plan usable, except for the
 * cyclic selection, which visits every row (the solve then fails with RK_EINVAL). */
int rk_setup(const void *A, rk_dtype dt, const float *row_scale, int64_t m, int64_t n,
             int64_t lda, void *workspace, size_t ws_bytes, void *stream, rk_plan **out);

/* Synchronise `stream` and return the device-side result of the build (RK_OK or
 * RK_ESETUP); on success *T_out and *L_out (either may be NULL) receive T and L. */
int rk_plan_status(const rk_plan *plan, void *stream, uint64_t *T_out, int32_t *L_out);

/* Synchronise `stream` and return ||A||_F^2 of the plan's law: T 2^L, the sum of the integer
 * row weights (each ||A_i||^2 truncated to the law's bits: about 1e-8 relative below the
 * exact value for a Gaussian matrix).  Errors as rk_plan_status. */
int rk_plan_frobenius2(const rk_plan *plan, void *stream, double *fro2);

/* Device addresses of the plan's tables (any may be NULL): K (uint64, m), P (uint64, m),
 * thr64 (uint64, m), alias (uint32, m), inv (float32, m: 1/||A_i||^2; 0 for zero rows and
 * for rows with ||A_i||^2 outside [2^-126, 2^126)). */
int rk_plan_tables(const rk_plan *plan, const uint64_t **K, const uint64_t **P,
                   const uint64_t **thr64, const uint32_t **alias, const float **inv);

void rk_plan_destroy(rk_plan *plan);

/* ------------------------------------------------------------------------ */
/* Sampling: draw of worker `worker`, projection counter t, stream id s:    */
/* Philox4x32-10 (Salmon et al., SC'11) with key (seed lo, seed hi) and      */
/* counter (t lo, t hi, worker, s); u = r0 | r1 << 32, u2 = r2 | r3 << 32;   */
/* bucket c = floor(u m / 2^64); row = c if u2 < thr64_c else alias_c.       */
/* Worker gamma's j-th projection of round k uses t = k * alpha + j.         */
/* ------------------------------------------------------------------------ */

/* Test hook: out[k] = draw of (seed, worker, t0 + k, stream_id), k < count (device, uint32). */
int rk_sample_indices(const rk_plan *plan, uint64_t seed, uint32_t worker, uint32_t stream_id,
                      uint64_t t0, int64_t count, uint32_t *out, void *stream);

/* Test hook for every row selection: out[k] = row of worker `worker` of q at projection
 * t0 + k under `sampling` (rk_sampling).  RK_SAMPLE_BLOCKS draws with the same Philox
 * words: c = floor(u T_g / 2^64) with T_g the integer weight of the worker's block, and the
 * row is the one whose prefix interval [P_i, P_i + K_i) of the plan holds P_start + c (a
 * block of zero weight gives row m, and a solve with it fails with RK_EINVAL).
 * RK_SAMPLE_CYCLIC uses no random bits. */
int rk_sample_indices_ex(const rk_plan *plan, uint64_t seed, uint32_t worker, uint32_t q,
                         uint32_t stream_id, int sampling, uint64_t t0, int64_t count,
                         uint32_t *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Solve: RKAB, Section 3.4.1 and Algorithm 3.  Each of q workers starts a   */
/* round from v = x, applies `alpha` projections                            */
/*   v <- v + omega (b_i - <A_i, v>) / ||A_i||^2 A_i^T      (Eq. (alg))      */
/* with rows i drawn from Eq. (prob_line), and the round ends with          */
/*   x <- (1/q) sum_{gamma = 0}^{q-1} v_gamma   (a fixed order, every run).   */
/* alpha = 1 is RKA, Eq. (rka_uni_weights); q = 1 is RK.                     */
/* One persistent kernel runs all rounds: every worker is one CTA (or a      */
/* cluster of CTAs splitting x) that keeps its v on chip and streams the     */
/* sampled rows from HBM into a ring of shared-memory stages; RKA with more  */
/* workers than SMs gives each CTA a share of the workers, whose single      */
/* projections from x it sums (the same result, Eq. (rka_eq)).               */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace one solve with q workers needs: with r = min(q, twice the SM
 * count of the current device), about (r + 1) * ceil(n / 4) * 16 + 256 r bytes. */
size_t rk_solve_workspace_bytes(const rk_plan *plan, int q);

/* Run `rounds` rounds (fewer if the convergence criterion is met).
 *   b          device, m floats
 *   x0         device, n floats: starting point (may alias x)
 *   x          device, n floats: result
 *   q          workers: up to twice the SM count (one CTA per worker, two per SM beyond
 *              the SM count; RK_ENOTCORESIDENT beyond), any q >= 1 for alpha = 1 (RKA:
 *              more workers than SMs are spread over one CTA per SM).  Rows too long for
 *              two shared-memory stages of one CTA (beyond about 27000 float32 columns)
 *              run RKA only, with 1 <= q <= 64 (x split by columns over one CTA per SM:
 *              each CTA streams its chunk of every sampled row and the dot products are
 *              summed across the grid in a fixed order), or RKAB with cluster_size > 1;
 *              anything else on such rows gives RK_EINVAL
 *   alpha      projections per worker between averages, >= 1
 *   seed       Philox key
 *   opts       NULL for defaults
 *   workspace  device, >= rk_solve_workspace_bytes(plan, q), 256-byte aligned
 * Asynchronous on `stream`; results (rounds done, last metric, device status) are read
 * with rk_solve_status.  Calls that share a workspace must not overlap. */
int rkab_solve(const rk_plan *plan, const float *b, const float *x0, float *x, int q,
               int64_t alpha, int64_t rounds, uint64_t seed, const rk_opts *opts,
               void *workspace, size_t ws_bytes, void *stream);

/* Outcome of a solve as rkab_solve_noalloc reports it (same meaning as rk_solve_status). */
typedef struct {
    int32_t status;        /* RK_OK, RK_ETIMEOUT, RK_EDIVERGED or RK_ESETUP */
    int32_t reserved;
    int64_t rounds_done;   /* rounds completed */
    double last_metric;    /* criterion value at the last check, -1 if none */
} rk_solve_result;

/* Bytes of the fixed device scratch array used by rkab_solve_noalloc. */
#define RK_NOALLOC_SCRATCH_BYTES (8u << 20)

/* rkab_solve for callers that cannot allocate device memory: a plugin or callback
 * hosted by another runtime that owns every device allocation and gives it only a
 * stream, or a real-time loop that forbids allocation after start-up.  The paper has
 * no counterpart; it is the same solve as rkab_solve (same kernel, same results) with
 * its scratch -- the run-state header, the q x n worker displacements, the
 * averaged iterate and the per-worker check partials -- in one file-scope device array of RK_NOALLOC_SCRATCH_BYTES
 * (8 MiB) instead of a caller workspace, so it allocates nothing.
 *   plan, b, x0, x, q, alpha, rounds, seed, opts   as for rkab_solve
 *   result   where the outcome is written when the solve ends (stream-ordered): any
 *            address cudaMemcpyAsync accepts (device or pinned host); NULL to skip
 * Options are checked as for rkab_solve (RK_EINVAL).  Returns RK_ETOOLARGE, before any
 * device work, when the scratch of this launch exceeds the array: about
 * (r + 1) * ceil(n / 4) * 16 + 256 r bytes with r = q, or r = the SM count for RKA
 * (alpha = 1) with more workers than SMs (at n = 10000 on 152 SMs: q <= 207 for
 * alpha > 1, any q for alpha = 1).  Every GPU that loads the library holds the array
 * until the process exits.  The first call on a device looks up the array's device
 * address with that device current and keeps it for the life of the process; make
 * that first call before any stream capture, and make no call after cudaDeviceReset.
 * All calls on a device share the array and it keeps the last call's contents (each
 * call clears the run-state header): calls whose work overlaps on the GPU race on it. */
int rkab_solve_noalloc(const rk_plan *plan, const float *b, const float *x0, float *x, int q,
                       int64_t alpha, int64_t rounds, uint64_t seed, const rk_opts *opts,
                       rk_solve_result *result, void *stream);

/* rkab_solve with alpha = 1 (RKA of Algorithm 1, Eq. (rka_uni_weights)). */
int rka_solve(const rk_plan *plan, const float *b, const float *x0, float *x, int q,
              int64_t rounds, uint64_t seed, const rk_opts *opts, void *workspace,
              size_t ws_bytes, void *stream);

/* Synchronise `stream` and read the outcome of the last solve that used `workspace`:
 * returns its device status (RK_OK, RK_ETIMEOUT, RK_EDIVERGED); *rounds_done and
 * *last_metric (criterion value at the last check, -1 if none) may be NULL. */
int rk_solve_status(const void *workspace, void *stream, int64_t *rounds_done,
                    double *last_metric);

/* ------------------------------------------------------------------------ */
/* Precision form: rows stored in BF16 or FP8 e4m3 (per-row float32 scale)   */
/* halve or quarter the bytes per projection; outer iterative refinement    */
/* with the float32 master A and float64-accumulated residuals wins back   */
/* the accuracy.  Not in the paper (whose precision is unstated); the inner */
/* solves are RKAB (Section 3.4.1) on the stored rows.                       */
/* ------------------------------------------------------------------------ */

/* Quantise A (device float32, m x n, lda) into out (device, m x ldo elements of dt):
 *   RK_BF16     out_ij = bf16 round-to-nearest-even of a_ij
 *   RK_FP8E4M3  s_i = max_j |a_ij| / 448 in float32 (1 for an all-zero row), written to
 *               row_scale[i] (device, m floats); out_ij = e4m3 round-to-nearest-even of
 *               a_ij / s_i, saturating to +-448 (OCP finite-only variant)
 * Columns n .. ldo-1 of out are zeroed.  ldo * element size must be a multiple of 16.
 * Asynchronous on `stream`. */
int rk_quantize(const float *A, int64_t m, int64_t n, int64_t lda, rk_dtype dt, void *out,
                int64_t ldo, float *row_scale, void *stream);

/* Bytes of device workspace rkab_refine needs for the stored-row plan and q workers. */
size_t rk_refine_workspace_bytes(const rk_plan *lowp, int q);

/* Iterative refinement of Ax = b.  x starts at x0 (may alias x); for outer = 0, 1, ...:
 *   r = b - A32 x               (float32 master rows, float64 accumulation, rounded to float32)
 *   d = RKAB on the rows of `lowp` for A~ d = r from d = 0: q workers, alpha projections
 *       per round, inner_rounds rounds, Philox stream id 3 + (outer << 8), relaxation
 *       opts->omega
 *   x = x + d                   (float32)
 * and stops after max_outer steps or, with opts->criterion = 1, after the first step with
 * ||x - x_ref|| / ||x_ref|| < opts->tol; with that criterion and tol > 0 each inner solve also
 * checks x + d after every round and stops as soon as it meets the criterion (its reference is
 * x_ref - x, its tolerance tol ||x_ref|| / ||x_ref - x||), so the rounds to tolerance are
 * counted as for a plain solve.  Synchronises `stream` once per outer step to read
 * the inner solve's status and the criterion; returns RK_OK or the first error (device
 * status of an inner solve included).  *outer_done and *last_metric (may be NULL) receive
 * the steps done and the criterion after the last one (-1 without a criterion).
 *   lowp     plan of the stored copy (RK_BF16, RK_FP8E4M3, or RK_F32 for plain refinement)
 *   A32      device float32 master rows (m x n, lda32), the same system as lowp's rows
 *   workspace  device, >= rk_refine_workspace_bytes(lowp, q), 256-byte aligned */
int rkab_refine(const rk_plan *lowp, const float *A32, int64_t lda32, const float *b,
                const float *x0, float *x, int q, int64_t alpha, int64_t inner_rounds,
                int64_t max_outer, uint64_t seed, const rk_opts *opts, void *workspace,
                size_t ws_bytes, void *stream, int64_t *outer_done, double *last_metric);

/* ------------------------------------------------------------------------ */
/* Differentiation form: the adjoint of x = argmin ||A x - b|| (Eq.          */
/* (ls_system)) for a loss L(x).  From the normal equations,                 */
/*   grad_b = y,  grad_A = r g^T - y x^T,  r = b - A x,                      */
/* where y is the minimum-norm solution of A^T y = dL/dx -- the limit of     */
/* Kaczmarz started at y = 0 on the underdetermined system (Section 2.1) --  */
/* and g solves the consistent system A g = y (so g = (A^T A)^{-1} dL/dx).   */
/* ------------------------------------------------------------------------ */

/* At (device, n x ldt, ldt >= m, ldt * 4 a multiple of 16) <- A^T for A (device float32,
 * m x n, lda).  Asynchronous on `stream`. */
int rk_transpose(const float *A, int64_t m, int64_t n, int64_t lda, float *At, int64_t ldt,
                 void *stream);

/* G (device, m x n, ldg) <- r g^T - y x^T for device vectors r, y (m) and g, x (n): the
 * rank-2 gradient of A, written once.  Asynchronous on `stream`. */
int rk_rank2(const float *r, const float *g, const float *y, const float *x, int64_t m, int64_t n,
             float *G, int64_t ldg, void *stream);

/* Bytes of device workspace rkab_adjoint needs. */
size_t rk_adjoint_workspace_bytes(const rk_plan *plan_A, const rk_plan *plan_At, int q_t, int q);

/* Backward pass of the least-squares solve at the point x (device, n floats):
 *   plan_A   float32 plan of A (m x n); plan_At float32 plan of A^T (n x m, e.g. from
 *            rk_transpose); both must outlive the call
 *   b        device, m floats;  gx device, n floats: dL/dx at x
 *   y-solve  RKAB on A^T y = gx from y = 0: q_t workers, alpha_t, rounds_t, opts_t
 *            (Philox stream id 1; omega, cluster_size, lookahead and sampling honoured)
 *   g-solve  RKAB on A g = y from g = 0: q workers, alpha, rounds, opts (stream id 2)
 *   grad_b   device, m floats <- y;  g device, n floats <- g
 *   grad_A   device, m x n (ldg) <- r g^T - y x^T with r = b - A x (float64-accumulated)
 * Synchronises `stream` at the end and returns RK_OK or the first error (device status of
 * either solve included). */
int rkab_adjoint(const rk_plan *plan_A, const rk_plan *plan_At, const float *b, const float *x,
                 const float *gx, int q_t, int q, int64_t alpha_t, int64_t rounds_t, int64_t alpha,
                 int64_t rounds, uint64_t seed, const rk_opts *opts_t, const rk_opts *opts,
                 float *grad_b, float *g, float *grad_A, int64_t ldg, void *workspace,
                 size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Residual of Eq. (system) / Eq. (ls_system) with float32 A and float64     */
/* accumulation:  r = b - A x,  ||r||_2  and  ||A^T r||_2.                   */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace rk_residual needs. */
size_t rk_residual_workspace_bytes(int64_t m, int64_t n);

/*   A   device float32 rows (m x n, lda);  b device m floats;  x device n floats
 *   r   device m doubles (may be NULL)
 *   norms_out  device, 2 doubles: [||r||, ||A^T r||] (may be NULL; ||A^T r|| costs a
 *              second pass over A and is computed only when want_atr != 0)
 * Asynchronous on `stream`. */
int rk_residual(const float *A, int64_t m, int64_t n, int64_t lda, const float *b,
                const float *x, double *r, double *norms_out, int want_atr, void *workspace,
                size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Solve with a stopping rule that needs no reference solution (the          */
/* convergence checks of Section 3.1 on the residual r = b - A x):           */
/*   RK_CRIT_RESIDUAL  ||r|| / ||b||                  (consistent systems)    */
/*   RK_CRIT_NORMAL    ||A^T r|| / (||A||_F ||r||)    (least squares,         */
/*                     Eq. (ls_system); one more pass over A per check)       */
/* every check_every rounds, with the float64-class residual of rk_residual  */
/* on the float32 rows.                                                       */
/* ------------------------------------------------------------------------ */
typedef enum { RK_CRIT_RESIDUAL = 2, RK_CRIT_NORMAL = 3 } rk_residual_criterion;

/* Bytes of device workspace rkab_solve_residual needs. */
size_t rk_solve_residual_workspace_bytes(const rk_plan *plan, int q);

/* Rounds of rkab_solve (opts as there; its criterion, tol and check_every are not used)
 * in stretches of check_every rounds that continue one stream of draws (round0 advances),
 * each followed by the residual criterion; stops after the first check with
 * metric < tol, or after max_rounds.
 *   A32      device float32 rows of the same system (m x n, lda32); NULL uses the plan's
 *            rows (float32 plans only)
 *   x        device, n floats (may alias x0); the iterate after the last stretch
 * Synchronous (waits for `stream` after every stretch).  *rounds_done and *last_metric
 * (host, may be NULL) receive the rounds run and the last criterion value; returns RK_OK,
 * or the first error (device status of a stretch included). */
int rkab_solve_residual(const rk_plan *plan, const float *A32, int64_t lda32, const float *b,
                        const float *x0, float *x, int q, int64_t alpha, int64_t max_rounds,
                        int64_t check_every, uint64_t seed, const rk_opts *opts, int criterion,
                        double tol, void *workspace, size_t ws_bytes, void *stream,
                        int64_t *rounds_done, double *last_metric);

/* ------------------------------------------------------------------------ */
/* Optimal uniform weight of RKA (Section 2.3.1, Eq. (best_alpha)) for a      */
/* consistent system, from s_min = sigma_min^2 / ||A||_F^2 and               */
/* s_max = sigma_max^2 / ||A||_F^2:                                          */
/*   alpha* = q / (1 + (q-1) s_min)                 if s_max - s_min <= 1/(q-1) */
/*   alpha* = 2q / (1 + (q-1)(s_min + s_max))       otherwise                 */
/* (q = 1 gives 1).  RKA with weight alpha* is rka_solve with               */
/* opts->omega = alpha*.                                                      */
/* ------------------------------------------------------------------------ */

/* Eq. (best_alpha); returns 0 for q < 1 or s_min, s_max outside [0, 1]. */
double rk_alpha_star(int q, double s_min, double s_max);

/* Bytes of device workspace rk_spectrum needs for k Lanczos steps. */
size_t rk_spectrum_workspace_bytes(int64_t m, int64_t n, int k);

/* Estimates of the extreme squared singular values of A (sigma_min^2, sigma_max^2 over
 * the min(m, n) singular values) and ||A||_F^2 for device float32 A (m x n, lda; 16-byte
 * aligned rows): k steps (1 <= k <= 512, at most min(m, n) used) of the symmetric Lanczos
 * process with full reorthogonalisation in float64, from a start vector drawn with
 * Philox4x32-10 (key = seed).  For m >= n it runs on A^T A, each step one pass over A
 * (one round of the RKA kernel over all rows; two passes when the rows are too long for
 * it); for m < n on A A^T (the same nonzero eigenvalues without the n - m zero ones of
 * A^T A), each step an A^T u pass and an A y pass.  The end eigenvalues of the
 * tridiagonal matrix satisfy sigma_min^2 <= out[0] and out[1] <= sigma_max^2 up to
 * rounding (equality once the process spans the space, e.g. k >= min(m, n)).
 *   out   host, 3 doubles <- [sigma_min^2 estimate, sigma_max^2 estimate, ||A||_F^2]
 *   steps_done  host (may be NULL) <- Lanczos steps taken (fewer than k on breakdown)
 *   workspace   device, >= rk_spectrum_workspace_bytes(m, n, k), 256-byte aligned
 * Synchronous: waits for `stream` once per step. */
int rk_spectrum(const float *A, int64_t m, int64_t n, int64_t lda, int k, uint64_t seed,
                void *workspace, size_t ws_bytes, void *stream, double *out, int *steps_done);

/* rk_spectrum with ||A||_F^2 supplied by the caller (fro2 > 0), skipping its pass over A:
 * out[2] <- fro2.  A plan of A gives it as T 2^L (rk_plan_status), its exact-integer
 * sampling law, to about 1e-8 relative.  fro2 <= 0 computes it like rk_spectrum. */
int rk_spectrum_ex(const float *A, int64_t m, int64_t n, int64_t lda, int k, uint64_t seed,
                   double fro2, void *workspace, size_t ws_bytes, void *stream, double *out,
                   int *steps_done);

/* s_min = sigma_min^2 / ||A||_F^2 and s_max = sigma_max^2 / ||A||_F^2 of Eq. (best_alpha)
 * from the 3 doubles rk_spectrum writes (clamped to [0, 1]); either output may be NULL.
 * RK_EINVAL when ||A||_F^2 (spectrum[2]) is not positive and finite. */
int rk_spectrum_ratios(const double *spectrum, double *s_min, double *s_max);

/* alpha* of Eq. (best_alpha) for RKA with q workers on A: rk_spectrum_ex (k Lanczos steps,
 * fro2 as there; rk_plan_frobenius2 gives it from a plan of A), rk_spectrum_ratios and
 * rk_alpha_star in one call.
 *   alpha      host <- alpha*
 *   out        host, 5 doubles or NULL <- [sigma_min^2, sigma_max^2, ||A||_F^2, s_min, s_max]
 *   steps_done host or NULL <- Lanczos steps taken
 *   workspace  device, >= rk_spectrum_workspace_bytes(m, n, k), 256-byte aligned
 * Synchronous, like rk_spectrum.  RK_EINVAL for q < 1 or a zero matrix. */
int rk_optimal_weight(const float *A, int64_t m, int64_t n, int64_t lda, int q, int k,
                      uint64_t seed, double fro2, void *workspace, size_t ws_bytes, void *stream,
                      double *alpha, double *out, int *steps_done);

/* Bytes of device workspace rk_partial_alpha_star needs. */
size_t rk_partial_alpha_workspace_bytes(int64_t m, int64_t n, int q, int k);

/* The Partial Matrix alpha of Section 3.3.1 (Table 1): for each worker g of q, alpha* of
 * Eq. (best_alpha) with q workers and s_min, s_max of its own row block A_g (rows
 * floor(g m / q) .. floor((g+1) m / q) - 1, the blocks of the Distributed Approach),
 * s = sigma^2(A_g) / ||A_g||_F^2, the extremes estimated by rk_spectrum(A_g, k, seed).
 * Pass the weights to rk_opts.worker_weight (after copying them to the device).
 *   weights  host, q floats <- the per-worker alpha
 *   spectra  host, 3 q doubles or NULL <- rk_spectrum's out[] of every block
 * RK_EINVAL when q < 1 or q > m (an empty block).  Synchronous, like rk_spectrum. */
int rk_partial_alpha_star(const float *A, int64_t m, int64_t n, int64_t lda, int q, int k,
                          uint64_t seed, void *workspace, size_t ws_bytes, void *stream,
                          float *weights, double *spectra);

/* Name of an error code. */
const char *rk_strerror(int code);

/* Number of kernel launches this library has enqueued in this process (all entry points). */
uint64_t rk_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* RKAB_H */
