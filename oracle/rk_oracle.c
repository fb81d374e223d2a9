/*
 * rk_oracle.c -- plain, slow FP64 CPU oracle for Randomized Kaczmarz (RK),
 * Randomized Kaczmarz with Averaging (RKA) and its block variant (RKAB) of
 * Ferreira, Acebron, Monteiro, "Parallelization Strategies for the Randomized
 * Kaczmarz Algorithm on Large-Scale Dense Systems" (arXiv 2401.17474).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark load this file.  It shares no code, header, table
 * or constant generator with the CUDA library; both follow the same written
 * definitions, stated below with the passage each one restates.
 *
 * Every floating-point quantity of the method is computed in double, in the
 * plain sequential order of its definition.  Inputs A are FP32 values promoted
 * exactly to double.  Compile with -ffp-contract=off (no fused multiply-add).
 *
 * Contents
 *   orc_philox4x32_10   counter-based generator of Salmon et al. (SC'11)
 *   orc_row_weights     exact integer encoding of the sampling law, Eq. (prob_line)
 *   orc_alias_build     alias table of that law by the sweeping construction
 *   orc_sample_row      one draw from the law for (seed, worker, projection)
 *   orc_select_row      row choice of a worker under the three selections: the
 *                       law above, the row blocks of the Distributed Approach
 *                       (Section 3.3.1), the cyclic sweep (Section 2.1)
 *   orc_rk              RK, Eq. (alg) with rows drawn by Eq. (prob_line)
 *   orc_rka_formula     RKA iteration written as Eq. (rka_uni_weights)
 *   orc_rkab            RKAB (Section 3.4.1, Algorithm 3): q workers, alpha
 *                       projections each, then the average
 *   orc_rkab_ext        the same with a row selection, per-row weights w_i of
 *                       Eq. (rka_eq) and per-worker weights (the Partial Matrix
 *                       alpha of Section 3.3.1)
 *   orc_residual        r = b - A x, ||r||, ||A^T r||
 *   orc_bf16_rne        FP32 -> BF16 round-to-nearest-even
 *   orc_fp8e4m3_rne     FP32 -> FP8 e4m3 (OCP "fn" variant) round-to-nearest-even,
 *                       saturating to +-448
 */
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------- */
/* Philox4x32-10.  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11, Section 3: ten rounds of the two 32x32->64 bit   */
/* multiplications with the published multipliers, the round key bumped by   */
/* the two Weyl constants after each round.                                  */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Sampling law, Eq. (prob_line): P{i = l} = ||A_l||^2 / ||A||_F^2.          */
/*                                                                           */
/* Encoded with exact integers so that every implementation that follows the */
/* definition produces the same table whatever its summation order:          */
/*   e_i  : exponent with max_j |a_ij| = f * 2^e_i, f in [0.5, 1)            */
/*   R_i  = sum_j floor(a_ij^2 * 2^(102 - 2 e_i))      (exact, < 2^128)       */
/*          so ||A_i||^2 ~= R_i * 2^(2 e_i - 102)                           */
/*   h_i  = bitlength(R_i) + 2 e_i - 102,  H = max_i h_i over nonzero rows   */
/*   L    = H + ceil(log2 m) - 62                                            */
/*   K_i  = floor(R_i * 2^(2 e_i - 102 - L))   (a right shift; sum K_i < 2^62)*/
/*   T    = sum_i K_i                                                        */
/* Rows of A must be finite; an all-zero A has no law (error).               */
/* ------------------------------------------------------------------------- */
static int bitlen128(u128 v)
{
    int b = 0;
    while (v) { ++b; v >>= 1; }
    return b;
}

static int ceil_log2_i64(int64_t m)
{
    int c = 0;
    while (((int64_t)1 << c) < m) ++c;
    return c;
}

int orc_row_weights(const float *A, int64_t m, int64_t n, int64_t lda,
                    uint64_t *K, uint64_t *T_out, int32_t *L_out)
{
    if (m < 1 || n < 1 || lda < n || n >= ((int64_t)1 << 26) || m >= ((int64_t)1 << 31))
        return ORC_EINVAL;
    u128 *R = (u128 *)malloc(sizeof(u128) * (size_t)m);
    int *e = (int *)malloc(sizeof(int) * (size_t)m);
    if (!R || !e) { free(R); free(e); return ORC_ENOMEM; }
    /* rows are independent: they may be taken by several threads; H is their maximum */
    int have = 0, bad = 0, H = INT_MIN;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(max : H) reduction(| : have, bad)
#endif
    for (int64_t i = 0; i < m; ++i) {
        const float *a = A + i * lda;
        double amax = 0.0;
        int finite = 1;
        for (int64_t j = 0; j < n; ++j) {
            double v = fabs((double)a[j]);
            if (!isfinite(v)) finite = 0;
            else if (v > amax) amax = v;
        }
        R[i] = 0; e[i] = 0;
        if (!finite) { bad = 1; continue; }
        if (amax == 0.0) continue;
        int ei;
        frexp(amax, &ei);
        e[i] = ei;
        for (int64_t j = 0; j < n; ++j) {
            double sq = (double)a[j] * (double)a[j];          /* exact: 48-bit product */
            double scaled = ldexp(sq, 102 - 2 * ei);          /* exact power-of-two scale */
            R[i] += (u128)floor(scaled);
        }
        int h = bitlen128(R[i]) + 2 * ei - 102;
        if (h > H) H = h;
        have = 1;
    }
    if (bad || !have) { free(R); free(e); return ORC_EINVAL; }
    int L = H + ceil_log2_i64(m) - 62;
    uint64_t T = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (R[i] == 0) { K[i] = 0; continue; }
        int shift = L + 102 - 2 * e[i];
        if (shift < 0) { free(R); free(e); return ORC_EINVAL; }  /* cannot happen, see header */
        K[i] = shift >= 128 ? 0 : (uint64_t)(R[i] >> shift);
        T += K[i];
    }
    free(R); free(e);
    if (T == 0) return ORC_EINVAL;
    *T_out = T;
    *L_out = L;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Alias table of the law K_i / T (Walker's alias method), built by the      */
/* sweeping construction of Huebschle-Schneider and Sanders, "Parallel       */
/* Weighted Random Sampling" (ACM TOMS 2022): buckets of capacity T, item    */
/* masses S_i = m K_i; lights (S < T) and heavies (S > T) are each taken in  */
/* ascending index order; each light bucket is topped up by the current      */
/* heavy; a heavy whose residual drops below T is closed at once as a bucket */
/* of its own, topped up by the next heavy.  Items with S = T fill their own */
/* bucket.  All arithmetic is exact (128-bit integers).                      */
/*                                                                           */
/* Output per bucket i: thr64_i = floor(thr_i * 2^64 / T) (UINT64_MAX when   */
/* thr_i = T) and alias_i.  A draw takes bucket c = floor(u m / 2^64) and    */
/* keeps c when u2 < thr64_c, else alias_c.                                  */
/* ------------------------------------------------------------------------- */
int orc_alias_build(const uint64_t *K, int64_t m, uint64_t T, uint64_t *thr64, uint32_t *alias)
{
    if (m < 1 || T == 0) return ORC_EINVAL;
    u128 *S = (u128 *)malloc(sizeof(u128) * (size_t)m);
    u128 *thr = (u128 *)malloc(sizeof(u128) * (size_t)m);
    int64_t *lights = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int64_t *heavies = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!S || !thr || !lights || !heavies) {
        free(S); free(thr); free(lights); free(heavies); return ORC_ENOMEM;
    }
    int64_t nl = 0, nh = 0;
    u128 TT = (u128)T;
    for (int64_t i = 0; i < m; ++i) {
        S[i] = (u128)(uint64_t)m * (u128)K[i];
        if (S[i] < TT) lights[nl++] = i;
        else if (S[i] > TT) heavies[nh++] = i;
        else { thr[i] = TT; alias[i] = (uint32_t)i; }
    }
    int rc = ORC_OK;
    if (nh > 0) {
        int64_t hp = 0;
        int64_t j = heavies[0];
        u128 r = S[j];
        for (int64_t k = 0; k < nl && rc == ORC_OK; ++k) {
            int64_t i = lights[k];
            thr[i] = S[i];
            alias[i] = (uint32_t)j;
            r -= (TT - S[i]);
            while (r < TT) {
                if (hp + 1 >= nh) { rc = ORC_EINVAL; break; }  /* impossible for exact totals */
                int64_t jn = heavies[hp + 1];
                thr[j] = r;
                alias[j] = (uint32_t)jn;
                r = S[jn] - (TT - r);
                ++hp;
                j = jn;
            }
        }
        if (rc == ORC_OK && (r != TT || hp != nh - 1)) rc = ORC_EINVAL;
        if (rc == ORC_OK) { thr[j] = TT; alias[j] = (uint32_t)j; }
    } else if (nl > 0) {
        rc = ORC_EINVAL;
    }
    if (rc == ORC_OK) {
        for (int64_t i = 0; i < m; ++i) {
            if (thr[i] >= TT) thr64[i] = UINT64_MAX;
            else thr64[i] = (uint64_t)((thr[i] << 64) / TT);
        }
    }
    free(S); free(thr); free(lights); free(heavies);
    return rc;
}

/* One draw from the law for worker `worker`, projection counter t, stream id
 * `stream`: Philox counter (t lo, t hi, worker, stream), key (seed lo, seed hi);
 * u = r0 | r1 << 32 picks the bucket, u2 = r2 | r3 << 32 the side.           */
int64_t orc_sample_row(uint64_t seed, uint64_t t, uint32_t worker, uint32_t stream,
                       int64_t m, const uint64_t *thr64, const uint32_t *alias)
{
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), worker, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    uint64_t u = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
    uint64_t u2 = (uint64_t)r[2] | ((uint64_t)r[3] << 32);
    int64_t c = (int64_t)(((u128)u * (u128)(uint64_t)m) >> 64);
    return u2 < thr64[c] ? c : (int64_t)alias[c];
}

/* Row of worker g of q at projection counter t under a row selection:
 *   0  the whole law (orc_sample_row);
 *   1  the Distributed Approach (Section 3.3.1): worker g keeps to its block of
 *      rows [g m / q, (g+1) m / q) and draws row i of it with probability
 *      K_i / T_g, T_g = the block's sum of K.  The Philox words are those of
 *      orc_sample_row; c = floor(u T_g / 2^64) and the row is the one whose
 *      interval [S_i, S_i + K_i) holds S_start + c, with S the exclusive prefix
 *      sum of K (found by a plain scan).  Returns -1 for a block of weight 0;
 *   2  the cyclic sweep (Section 2.1): row (g m / q + t) mod m.                */
int64_t orc_select_row(int sampling, uint64_t seed, uint64_t t, uint32_t g, int q, uint32_t stream,
                       int64_t m, const uint64_t *thr64, const uint32_t *alias, const uint64_t *K)
{
    if (sampling == 0) return orc_sample_row(seed, t, g, stream, m, thr64, alias);
    int64_t start = (int64_t)(((u128)g * (u128)m) / (u128)q);
    int64_t end = (int64_t)(((u128)(g + 1) * (u128)m) / (u128)q);
    if (sampling == 2) return (int64_t)(((uint64_t)start + t) % (uint64_t)m);
    uint64_t tg = 0;
    for (int64_t i = start; i < end; ++i) tg += K[i];
    if (tg == 0) return -1;
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), g, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    uint64_t u = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
    uint64_t c = (uint64_t)(((u128)u * (u128)tg) >> 64);
    /* walk the block: the row whose share [acc, acc + K_i) of the block holds c */
    uint64_t acc = 0;
    for (int64_t i = start; i < end; ++i) {
        if (c < acc + K[i]) return i;
        acc += K[i];
    }
    return -1;
}

/* count consecutive row choices of worker g of q: out[k] = row at t = t0 + k. */
void orc_select_rows(int sampling, uint64_t seed, uint32_t g, int q, uint32_t stream, uint64_t t0,
                     int64_t count, int64_t m, const uint64_t *thr64, const uint32_t *alias,
                     const uint64_t *K, int64_t *out)
{
    for (int64_t k = 0; k < count; ++k)
        out[k] = orc_select_row(sampling, seed, t0 + (uint64_t)k, g, q, stream, m, thr64, alias, K);
}

/* count consecutive draws of one worker: out[k] = draw at t = t0 + k. */
void orc_sample_rows(uint64_t seed, uint32_t worker, uint32_t stream, uint64_t t0, int64_t count,
                     int64_t m, const uint64_t *thr64, const uint32_t *alias, int64_t *out)
{
    for (int64_t k = 0; k < count; ++k)
        out[k] = orc_sample_row(seed, t0 + (uint64_t)k, worker, stream, m, thr64, alias);
}

/* ------------------------------------------------------------------------- */
/* Plain helpers in double.                                                  */
/* ------------------------------------------------------------------------- */
static double row_dot(const float *a, const double *v, int64_t n)
{
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += (double)a[j] * v[j];
    return s;
}

static double row_norm2(const float *a, int64_t n)
{
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += (double)a[j] * (double)a[j];
    return s;
}

/* One Kaczmarz projection, Eq. (alg): v <- v + omega (b_i - <A_i, v>) / ||A_i||^2 A_i^T */
static void project(const float *a, double bi, double w, double omega, double *v, int64_t n)
{
    double rho = bi - row_dot(a, v, n);
    double s = omega * rho / w;
    for (int64_t j = 0; j < n; ++j) v[j] += s * (double)a[j];
}

static double rel_err(const double *x, const double *xr, int64_t n)
{
    double d = 0.0, r = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double e = x[j] - xr[j];
        d += e * e;
        r += xr[j] * xr[j];
    }
    return sqrt(d) / sqrt(r);
}

/* Row norms ||A_i||^2 in double, plain sequential sums. */
void orc_row_norms(const float *A, int64_t m, int64_t n, int64_t lda, double *w)
{
    for (int64_t i = 0; i < m; ++i) w[i] = row_norm2(A + i * lda, n);
}

/* ------------------------------------------------------------------------- */
/* RK: Eq. (alg) with row i drawn from Eq. (prob_line) (Section 2.2).        */
/* Projection k uses the draw of (worker, t = t0 + k).                       */
/* ------------------------------------------------------------------------- */
int orc_rk(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
           const double *x0, double *x, int64_t iters, int64_t t0, uint64_t seed,
           uint32_t worker, uint32_t stream, double omega,
           const uint64_t *thr64, const uint32_t *alias)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)m);
    if (!w) return ORC_ENOMEM;
    orc_row_norms(A, m, n, lda, w);
    if (x != x0) memcpy(x, x0, sizeof(double) * (size_t)n);
    for (int64_t k = 0; k < iters; ++k) {
        int64_t i = orc_sample_row(seed, (uint64_t)(t0 + k), worker, stream, m, thr64, alias);
        project(A + i * lda, b[i], w[i], omega, x, n);
    }
    free(w);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* RKA written as Eq. (rka_uni_weights):                                     */
/*   x_{k+1} = x_k + (omega/q) sum_{i in tau_k} (b_i - <A_i, x_k>)/||A_i||^2 A_i^T */
/* with tau_k the q draws of workers 0..q-1 at projection counter k.         */
/* ------------------------------------------------------------------------- */
int orc_rka_formula(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                    const double *x0, double *x, int q, int64_t iters, uint64_t seed,
                    uint32_t stream, double omega, const uint64_t *thr64, const uint32_t *alias)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)m);
    double *acc = (double *)malloc(sizeof(double) * (size_t)n);
    if (!w || !acc) { free(w); free(acc); return ORC_ENOMEM; }
    orc_row_norms(A, m, n, lda, w);
    if (x != x0) memcpy(x, x0, sizeof(double) * (size_t)n);
    for (int64_t k = 0; k < iters; ++k) {
        for (int64_t j = 0; j < n; ++j) acc[j] = 0.0;
        for (int g = 0; g < q; ++g) {
            int64_t i = orc_sample_row(seed, (uint64_t)k, (uint32_t)g, stream, m, thr64, alias);
            const float *a = A + i * lda;
            double coef = (b[i] - row_dot(a, x, n)) / w[i];
            for (int64_t j = 0; j < n; ++j) acc[j] += coef * (double)a[j];
        }
        for (int64_t j = 0; j < n; ++j) x[j] += (omega / (double)q) * acc[j];
    }
    free(w); free(acc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* RKAB, Section 3.4.1 and Algorithm 3: in each round every worker gamma     */
/* starts from v_gamma = x, applies `alpha` projections of Eq. (alg) with    */
/* its own draws (projection counter t = round * alpha + j), and then        */
/* x <- (1/q) sum_gamma v_gamma, summed in the order gamma = 0 .. q-1.       */
/* alpha = 1 is RKA; q = 1 is RK.                                             */
/*                                                                           */
/* round0 shifts the projection counter (resume).  same_stream != 0 gives    */
/* every worker the draws of worker 0.  When x_ref != NULL and tol > 0 the   */
/* run stops after the first average with ||x - x_ref|| / ||x_ref|| < tol.   */
/* trace (optional, rounds entries) receives that relative error after each  */
/* average when x_ref != NULL.  Workers run in parallel on `threads` OpenMP  */
/* threads (the shared-memory structure of Algorithm 3); the result does not */
/* depend on the thread count.                                              */
/*                                                                           */
/* Weights: a projection of row i by worker gamma uses the relaxation        */
/* omega * w_i * u_gamma, w_i = row_weight[i] (Eq. (rka_eq)), u_gamma =      */
/* worker_weight[gamma] (a per-thread alpha, Section 3.3.1); NULL means 1.   */
/* ------------------------------------------------------------------------- */
int orc_rkab_ext(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                 const double *x0, double *x, int q, int64_t alpha, int64_t rounds,
                 int64_t round0, uint64_t seed, uint32_t stream, double omega,
                 const uint64_t *thr64, const uint32_t *alias, int same_stream, int threads,
                 const double *x_ref, double tol, int64_t *rounds_done, double *trace,
                 int sampling, const uint64_t *K, const double *row_weight,
                 const double *worker_weight)
{
    if (q < 1 || alpha < 1 || rounds < 0) return ORC_EINVAL;
    if (sampling != 0 && (same_stream || (sampling == 1 && !K))) return ORC_EINVAL;
    double *w = (double *)malloc(sizeof(double) * (size_t)m);
    double *V = (double *)malloc(sizeof(double) * (size_t)q * (size_t)n);
    if (!w || !V) { free(w); free(V); return ORC_ENOMEM; }
    orc_row_norms(A, m, n, lda, w);
    if (x != x0) memcpy(x, x0, sizeof(double) * (size_t)n);
    if (threads < 1) threads = 1;
    int64_t done = 0;
    for (int64_t r = 0; r < rounds; ++r) {
        int64_t round = round0 + r;
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
        for (int g = 0; g < q; ++g) {
            double *v = V + (size_t)g * (size_t)n;
            memcpy(v, x, sizeof(double) * (size_t)n);
            uint32_t worker = same_stream ? 0u : (uint32_t)g;
            double ug = worker_weight ? worker_weight[g] : 1.0;
            for (int64_t j = 0; j < alpha; ++j) {
                uint64_t t = (uint64_t)(round * alpha + j);
                int64_t i = orc_select_row(sampling, seed, t, worker, q, stream, m, thr64, alias, K);
                if (i < 0) continue;   /* a block of weight 0 (reported by the caller) */
                double wi = row_weight ? row_weight[i] : 1.0;
                project(A + i * lda, b[i], w[i], omega * wi * ug, v, n);
            }
        }
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int g = 0; g < q; ++g) s += V[(size_t)g * (size_t)n + (size_t)j];
            x[j] = s / (double)q;
        }
        done = r + 1;
        if (x_ref) {
            double e = rel_err(x, x_ref, n);
            if (trace) trace[r] = e;
            if (tol > 0.0 && e < tol) break;
        }
    }
    if (rounds_done) *rounds_done = done;
    free(w); free(V);
    return ORC_OK;
}

/* RKAB with the whole law and unit weights. */
int orc_rkab(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
             const double *x0, double *x, int q, int64_t alpha, int64_t rounds,
             int64_t round0, uint64_t seed, uint32_t stream, double omega,
             const uint64_t *thr64, const uint32_t *alias, int same_stream, int threads,
             const double *x_ref, double tol, int64_t *rounds_done, double *trace)
{
    return orc_rkab_ext(A, m, n, lda, b, x0, x, q, alpha, rounds, round0, seed, stream, omega,
                        thr64, alias, same_stream, threads, x_ref, tol, rounds_done, trace, 0,
                        NULL, NULL, NULL);
}

/* Worker iterates of one RKAB round (before the average), for the Jensen
 * check of the averaging step: V (q x n) receives v_gamma.                  */
int orc_rkab_round_workers(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                           const double *x, double *V, int q, int64_t alpha, int64_t round,
                           uint64_t seed, uint32_t stream, double omega,
                           const uint64_t *thr64, const uint32_t *alias)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)m);
    if (!w) return ORC_ENOMEM;
    orc_row_norms(A, m, n, lda, w);
    for (int g = 0; g < q; ++g) {
        double *v = V + (size_t)g * (size_t)n;
        memcpy(v, x, sizeof(double) * (size_t)n);
        for (int64_t j = 0; j < alpha; ++j) {
            uint64_t t = (uint64_t)(round * alpha + j);
            int64_t i = orc_sample_row(seed, t, (uint32_t)g, stream, m, thr64, alias);
            project(A + i * lda, b[i], w[i], omega, v, n);
        }
    }
    free(w);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Residual of Eq. (system) / Eq. (ls_system): r = b - A x, ||r|| and        */
/* ||A^T r|| (the normal-equation residual), all in double.  r may be NULL.  */
/* ------------------------------------------------------------------------- */
int orc_residual(const float *A, int64_t m, int64_t n, int64_t lda, const double *b,
                 const double *x, double *r, double *rnorm, double *atr_norm)
{
    double *atr = (double *)calloc((size_t)n, sizeof(double));
    if (!atr) return ORC_ENOMEM;
    double rr = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const float *a = A + i * lda;
        double ri = b[i] - row_dot(a, x, n);
        if (r) r[i] = ri;
        rr += ri * ri;
        for (int64_t j = 0; j < n; ++j) atr[j] += ri * (double)a[j];
    }
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += atr[j] * atr[j];
    if (rnorm) *rnorm = sqrt(rr);
    if (atr_norm) *atr_norm = sqrt(s);
    free(atr);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Stored-row precisions.                                                    */
/* BF16: the upper 16 bits of the FP32 pattern after round-to-nearest-even.  */
/* ------------------------------------------------------------------------- */
uint16_t orc_bf16_rne(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) {            /* inf or nan */
        if (u & 0x007FFFFFu) return (uint16_t)((u >> 16) | 0x0040u);
        return (uint16_t)(u >> 16);
    }
    uint32_t lsb = (u >> 16) & 1u;
    uint32_t rounded = u + 0x7FFFu + lsb;
    return (uint16_t)(rounded >> 16);
}

/* Value of an FP8 e4m3 ("fn": no infinities, 0x7F/0xFF NaN) code. */
double orc_fp8e4m3_value(uint8_t c)
{
    int s = c >> 7, e = (c >> 3) & 0xF, f = c & 7;
    double v;
    if (e == 0xF && f == 7) return NAN;
    if (e == 0) v = ldexp((double)f, -9);               /* subnormal: f/8 * 2^-6 */
    else v = ldexp(1.0 + f / 8.0, e - 7);
    return s ? -v : v;
}

/* FP32 -> e4m3 by brute force: the representable value nearest to f, ties to
 * the even code (last mantissa bit 0), values beyond 448 saturate to +-448.  */
uint8_t orc_fp8e4m3_rne(float f)
{
    double x = (double)f;
    if (isnan(x)) return 0x7F;
    uint8_t sign = (x < 0.0 || (x == 0.0 && signbit(x))) ? 0x80 : 0x00;
    double ax = fabs(x);
    if (ax >= 448.0) return (uint8_t)(sign | 0x7E);
    uint8_t best = 0;
    double bestd = INFINITY;
    for (int c = 0; c <= 0x7E; ++c) {
        double d = fabs(orc_fp8e4m3_value((uint8_t)c) - ax);
        if (d < bestd || (d == bestd && (c & 1) == 0)) { bestd = d; best = (uint8_t)c; }
    }
    return (uint8_t)(sign | best);
}
