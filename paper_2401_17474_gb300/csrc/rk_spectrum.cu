// rk_spectrum.cu -- the spectrum that the optimal uniform weight of RKA needs
// (Eq. (best_alpha): s_min = sigma_min^2 / ||A||_F^2, s_max = sigma_max^2 / ||A||_F^2).
// The extreme eigenvalues of A^T A are estimated by k steps of the symmetric
// Lanczos process on A^T A with full reorthogonalisation (classical Gram-Schmidt
// applied twice per step) in FP64 vectors; the operator is applied as two passes
// over A by the residual kernels (r = -A v, then A^T r).  The end eigenvalues of
// the k x k tridiagonal matrix are found on the host by Sturm-sequence bisection.
// Ritz values lie inside the spectrum, so lambda_min <= est_min and
// est_max <= lambda_max (up to rounding): with est_min, the weight of
// Eq. (best_alpha) errs on the small side.
// A^T A v is applied in one pass over A where the solve kernel can hold a row
// (n up to 20480): one round of the RKA kernel in which every row is taken once
// (cyclic selection, q = m workers), with b = 0, unit reciprocal norms and the
// weight -m, returns v + A^T A v in float32.  Longer rows take the two residual
// passes (float64-class).  For m < n the process runs on A A^T in R^m instead (the
// same nonzero eigenvalues, without the n - m zero eigenvalues of A^T A): each step
// is the A^T r pass (y = -A^T v) and the row pass (-A y).
#include <cmath>
#include <cstdint>
#include <vector>

#include "rk_common.cuh"
#include "rk_internal.h"

namespace rk {

constexpr int kSpThreads = 256;
constexpr uint32_t kSpStream = 0x5EC7u;   // Philox stream id of the start vector

// v_j uniform in [-1, 1): Philox4x32-10 at counter (j, 0, stream), key = seed,
// the top 53 bits of the first 64-bit word.
__global__ void lanczos_start_kernel(double* __restrict__ v, int64_t n, uint64_t seed) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const U4 r = philox10(U4{(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 0u, kSpStream},
                              (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint64_t u = (uint64_t)r.x | ((uint64_t)r.y << 32);
        v[j] = 2.0 * ((double)(u >> 11) * 0x1.0p-53) - 1.0;
    }
}

// Fixed-order block sum of the threads' partials (power-of-two tree).
__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kSpThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// c[i] = <w, V_i> for i < cnt (one block per i).
__global__ void __launch_bounds__(kSpThreads) multi_dot_kernel(const double* __restrict__ V, int64_t ldv,
                                                               const double* __restrict__ w, int64_t n,
                                                               double* __restrict__ c) {
    __shared__ double sh[kSpThreads];
    const double* vi = V + (size_t)blockIdx.x * (size_t)ldv;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += kSpThreads) acc = fma(w[j], vi[j], acc);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) c[blockIdx.x] = s;
}

// w_j -= sum_{i < cnt} c_i V_ij (ascending i).
__global__ void multi_sub_kernel(double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int cnt,
                                 const double* __restrict__ c, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double s = w[j];
        for (int i = 0; i < cnt; ++i) s = fma(-c[i], V[(size_t)i * (size_t)ldv + j], s);
        w[j] = s;
    }
}

// out[0] = ||w||^2 (one block).
__global__ void __launch_bounds__(kSpThreads) norm2_kernel(const double* __restrict__ w, int64_t n,
                                                           double* __restrict__ out) {
    __shared__ double sh[kSpThreads];
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += kSpThreads) acc = fma(w[j], w[j], acc);
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = s;
}

// vnext = w / sqrt(nrm2[0]) (zero when w is zero), vf = float(vnext).
__global__ void scale_kernel(const double* __restrict__ w, int64_t n, const double* __restrict__ nrm2,
                             double* __restrict__ vnext, float* __restrict__ vf) {
    const double nn = nrm2[0];
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double t = w[j] * inv;
        vnext[j] = t;
        vf[j] = (float)t;
    }
}

// a^2 added to the compensated float32 pair (hi, lo): a a = p + e exactly
// (e = fma(a, a, -p)), p by TwoSum.
__device__ __forceinline__ void add_square(float& hi, float& lo, float t) {
    const float p = __fmul_rn(t, t);
    const float e = fmaf(t, t, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// Per-block partial sums of a_ij^2: one warp per row, each lane reading float4
// slices (four in flight) and accumulating the exact squares in two compensated
// float32 pairs (TwoSum; about 2^-46 relative), the pairs combined in FP64 per
// block.  The FP64 pipe of the device is slow, so no FP64 operation runs per
// element.  Rows are 16-byte aligned (lda a multiple of 4).
__global__ void __launch_bounds__(kSpThreads) fro_rows_kernel(const float* __restrict__ A, int64_t m,
                                                              int64_t n, int64_t lda,
                                                              double* __restrict__ part) {
    __shared__ double sh[kSpThreads];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    const int64_t n4 = n / 4;
    for (int64_t i = (int64_t)blockIdx.x * (kSpThreads / 32) + warp; i < m;
         i += (int64_t)gridDim.x * (kSpThreads / 32)) {
        const float* a = A + i * lda;
        const float4* a4 = reinterpret_cast<const float4*>(a);
#pragma unroll 4
        for (int64_t c = lane; c < n4; c += 32) {
            const float4 v = __ldcs(a4 + c);
            add_square(h0, l0, v.x);
            add_square(h1, l1, v.y);
            add_square(h0, l0, v.z);
            add_square(h1, l1, v.w);
        }
        for (int64_t j = n4 * 4 + lane; j < n; j += 32) add_square(h0, l0, __ldcs(a + j));
    }
    const double s = block_sum(((double)h0 + (double)l0) + ((double)h1 + (double)l1), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[0] = sum of the partials in block order.
__global__ void sum_parts_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < nb; ++k) s += part[k];
        out[0] = s;
    }
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with diagonal
// a[0..s) and squared off-diagonals b2[1..s) (b2[i] couples i-1 and i): the
// count of negative pivots of the LDL^T factorisation of T - x I (Sylvester's
// law of inertia); tiny pivots are replaced by -pivmin.
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b2, double x,
                       double pivmin) {
    int cnt = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        d = (a[i] - x) - (i ? b2[i] / d : 0.0);
        if (std::fabs(d) < pivmin) d = -pivmin;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Smallest and largest eigenvalue of the tridiagonal matrix by bisection inside
// the Gershgorin interval.
static void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double* lmin,
                             double* lmax) {
    const size_t s = a.size();
    std::vector<double> b2(s, 0.0);
    double lo = INFINITY, hi = -INFINITY, scale = 0.0;
    for (size_t i = 0; i < s; ++i) {
        const double r = (i ? std::fabs(b[i]) : 0.0) + (i + 1 < s ? std::fabs(b[i + 1]) : 0.0);
        lo = std::fmin(lo, a[i] - r);
        hi = std::fmax(hi, a[i] + r);
        if (i) b2[i] = b[i] * b[i];
        scale = std::fmax(scale, std::fabs(a[i]) + r);
    }
    const double pivmin = std::fmax(scale, 1e-300) * 1e-300;
    const int ss = (int)s;
    auto bisect = [&](int k) {   // smallest x with count(x) >= k, i.e. the k-th eigenvalue
        double l = lo - 1e-12 * scale, h = hi + 1e-12 * scale;
        for (int it = 0; it < 200 && h - l > 2e-16 * std::fmax(std::fabs(l), std::fabs(h)); ++it) {
            const double mid = 0.5 * (l + h);
            if (sturm_count(a, b2, mid, pivmin) >= k) h = mid;
            else l = mid;
        }
        return 0.5 * (l + h);
    };
    *lmin = bisect(1);
    *lmax = bisect(ss);
}

struct SpecWs {
    double* scal;    // [0] ||w||^2, [1] ||A||_F^2
    double* c1;      // k + 1
    double* c2;      // k + 1
    double* V;       // (k + 1) x ldv
    int64_t ldv;
    double* w;       // n
    float* vf;       // n
    double* fpart;   // fro partials
    void* res;       // residual workspace (two-pass operator)
    SetupInfo* sinfo;  // a passed plan status for the one-pass operator
    float* ones;     // m
    float* zeros;    // m
    float* vout;     // n: v + A^T A v
    void* solve;     // solve workspace of the one-pass operator
};

static int fro_blocks(int64_t m) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (m + (kSpThreads / 32) - 1) / (kSpThreads / 32);
    const int64_t cap = (int64_t)sms * 4;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

static SpecWs spec_carve(void* base, int64_t m, int64_t n, int k) {
    uint8_t* p = static_cast<uint8_t*>(base);
    SpecWs w;
    w.ldv = (n + 31) / 32 * 32;
    w.scal = reinterpret_cast<double*>(p);
    p += 256;
    w.c1 = reinterpret_cast<double*>(p);
    p += align256((size_t)(k + 1) * 8);
    w.c2 = reinterpret_cast<double*>(p);
    p += align256((size_t)(k + 1) * 8);
    w.V = reinterpret_cast<double*>(p);
    p += align256((size_t)(k + 1) * (size_t)w.ldv * 8);
    w.w = reinterpret_cast<double*>(p);
    p += align256((size_t)n * 8);
    w.vf = reinterpret_cast<float*>(p);
    p += align256((size_t)n * 4);
    w.fpart = reinterpret_cast<double*>(p);
    p += align256((size_t)fro_blocks(m) * 8);
    w.res = p;
    p += align256(residual_ws_bytes(m, n));
    w.sinfo = reinterpret_cast<SetupInfo*>(p);
    p += 256;
    w.ones = reinterpret_cast<float*>(p);
    p += align256((size_t)m * 4);
    w.zeros = reinterpret_cast<float*>(p);
    p += align256((size_t)m * 4);
    w.vout = reinterpret_cast<float*>(p);
    p += align256((size_t)n * 4);
    w.solve = p;
    return w;
}

static size_t one_pass_solve_bytes(int64_t m, int64_t n) {
    Plan pl{};
    pl.n = n;
    pl.m = m;
    return solve_ws_bytes(&pl, (int)m);
}

size_t spectrum_ws_bytes(int64_t m, int64_t n, int k) {
    const size_t ldv = (size_t)((n + 31) / 32 * 32);
    return 256 + 2 * align256((size_t)(k + 1) * 8) + align256((size_t)(k + 1) * ldv * 8) +
           align256((size_t)n * 8) + align256((size_t)n * 4) + align256((size_t)fro_blocks(m) * 8) +
           align256(residual_ws_bytes(m, n)) + 256 + 2 * align256((size_t)m * 4) +
           align256((size_t)n * 4) + one_pass_solve_bytes(m, n);
}

__global__ void fill_kernel(float* __restrict__ a, int64_t m, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void to_float_kernel(const double* __restrict__ y, int64_t n, float* __restrict__ yf) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        yf[j] = (float)y[j];
}

// w = vout - v in float64 (vout = v + A^T A v from the one-pass operator).
__global__ void diff_kernel(const float* __restrict__ vout, const float* __restrict__ v, int64_t n,
                            double* __restrict__ w) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        w[j] = (double)vout[j] - (double)v[j];
}

// w = A^T A v by one round of the RKA kernel over every row (see the head of this
// file); returns RK_EINVAL when no solve variant holds a row of n columns.
static int one_pass_normal_matvec(const Plan& pl, const SpecWs& w, int64_t n, cudaStream_t st) {
    SolveArgs a;
    a.plan = &pl;
    a.b = w.zeros;
    a.x0 = w.vf;
    a.x = w.vout;
    a.q = (int)pl.m;
    a.alpha = 1;
    a.rounds = 1;
    a.seed = 0;
    rk_opts_default(&a.opts);
    a.opts.omega = -(float)pl.m;   // c_i = m <A_i, v>, averaged over the m workers
    a.opts.check_every = 0;
    a.opts.sampling = RK_SAMPLE_CYCLIC;   // worker i takes row i
    a.info = static_cast<SolveInfo*>(w.solve);
    a.ldv = (n + 3) / 4 * 4;
    a.V = reinterpret_cast<float*>(static_cast<uint8_t*>(w.solve) + align256(sizeof(SolveInfo)));
    if (cudaMemsetAsync(a.info, 0, sizeof(SolveInfo), st) != cudaSuccess) return RK_ECUDA;
    const int rc = launch_solve(a, st);
    if (rc != RK_OK) return rc;
    diff_kernel<<<(unsigned)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048), 256, 0, st>>>(w.vout, w.vf,
                                                                                              n, w.w);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

static int grid_for(int64_t n) {
    const int64_t g = (n + kSpThreads - 1) / kSpThreads;
    return (int)(g < 1 ? 1 : (g < 2048 ? g : 2048));
}

int run_spectrum(const float* A, int64_t m, int64_t n, int64_t lda, int k, uint64_t seed, void* ws,
                 cudaStream_t st, double* out, int* steps_done, double fro2_known) {
    SpecWs w = spec_carve(ws, m, n, k);
    if (steps_done) *steps_done = 0;
    // ||A||_F^2, unless the caller knows it
    if (!(fro2_known > 0.0)) {
        const int fb = fro_blocks(m);
        fro_rows_kernel<<<fb, kSpThreads, 0, st>>>(A, m, n, lda, w.fpart);
        sum_parts_kernel<<<1, 32, 0, st>>>(w.fpart, fb, w.scal + 1);
        count_launch(2);
    }
    // the process runs on A^T A in R^n, or for m < n on A A^T in R^m: the same nonzero
    // eigenvalues without the n - m zero ones, which rounding would otherwise bring in
    // (a well separated end of the spectrum, found within a few steps)
    const bool wide = m < n;
    const int64_t d = wide ? m : n;
    // v_0: seeded start vector, normalised
    lanczos_start_kernel<<<grid_for(d), kSpThreads, 0, st>>>(w.w, d, seed);
    norm2_kernel<<<1, kSpThreads, 0, st>>>(w.w, d, w.scal);
    scale_kernel<<<grid_for(d), kSpThreads, 0, st>>>(w.w, d, w.scal, w.V, w.vf);
    count_launch(3);
    if (cudaGetLastError() != cudaSuccess) return RK_ECUDA;

    // the plan of the one-pass operator: rows of A, unit reciprocal norms, a passed status
    Plan pl{};
    pl.A = A;
    pl.dt = RK_F32;
    pl.row_scale = nullptr;
    pl.m = m;
    pl.n = n;
    pl.lda = lda;
    pl.ws.info = w.sinfo;
    pl.ws.inv = w.ones;
    if (cudaMemsetAsync(w.sinfo, 0, 256, st) != cudaSuccess) return RK_ECUDA;
    fill_kernel<<<grid_for(m), kSpThreads, 0, st>>>(w.ones, m, 1.0f);
    fill_kernel<<<grid_for(m), kSpThreads, 0, st>>>(w.zeros, m, 0.0f);
    count_launch(2);
    bool one_pass = m < (int64_t)1 << 31;

    std::vector<double> alpha, beta(1, 0.0);   // beta[j] couples steps j-1 and j
    double fro2 = 0.0;
    for (int j = 0; j < k; ++j) {
        int rc = RK_EINVAL;
        if (wide) {
            // w = A A^T v_j: y = -A^T v_j (n doubles, in w), its float32 copy, then -A y
            rc = launch_transpose_matvec(A, m, n, lda, w.V + (size_t)j * (size_t)w.ldv, w.w, w.res, st);
            if (rc != RK_OK) return rc;
            to_float_kernel<<<grid_for(n), kSpThreads, 0, st>>>(w.w, n, w.vout);
            count_launch();
            rc = launch_rows_matvec(A, m, n, lda, w.vout, w.w, w.res, st);
        } else {
            // w = A^T A v_j
            if (one_pass) {
                rc = one_pass_normal_matvec(pl, w, n, st);
                if (rc == RK_EINVAL) one_pass = false;   // rows too long for the solve kernel
            }
            if (!one_pass) rc = launch_normal_matvec(A, m, n, lda, w.vf, w.w, w.res, st);
        }
        if (rc != RK_OK) return rc;
        // two passes of classical Gram-Schmidt against v_0 .. v_j
        const int cnt = j + 1;
        multi_dot_kernel<<<cnt, kSpThreads, 0, st>>>(w.V, w.ldv, w.w, d, w.c1);
        multi_sub_kernel<<<grid_for(d), kSpThreads, 0, st>>>(w.w, w.V, w.ldv, cnt, w.c1, d);
        multi_dot_kernel<<<cnt, kSpThreads, 0, st>>>(w.V, w.ldv, w.w, d, w.c2);
        multi_sub_kernel<<<grid_for(d), kSpThreads, 0, st>>>(w.w, w.V, w.ldv, cnt, w.c2, d);
        norm2_kernel<<<1, kSpThreads, 0, st>>>(w.w, d, w.scal);
        scale_kernel<<<grid_for(d), kSpThreads, 0, st>>>(w.w, d, w.scal, w.V + (size_t)cnt * (size_t)w.ldv,
                                                         w.vf);
        count_launch(6);
        double h[4];
        int solve_status = 0;
        if (cudaMemcpyAsync(&h[0], w.c1 + j, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&h[1], w.c2 + j, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&h[2], w.scal, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            (!wide && one_pass && cudaMemcpyAsync(&solve_status, w.solve, sizeof(int),
                                                  cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RK_ECUDA;
        if (solve_status != 0) return solve_status;
        fro2 = h[3];
        if (!std::isfinite(h[0]) || !std::isfinite(h[2])) return RK_EDIVERGED;
        alpha.push_back(h[0] + h[1]);   // <A^T A v_j, v_j> with the second pass's correction
        const double bn = std::sqrt(h[2]);
        if (steps_done) *steps_done = j + 1;
        // an invariant subspace ends the process (always by j = d - 1)
        double amax = 0.0;
        for (double a : alpha) amax = std::fmax(amax, std::fabs(a));
        if (!(bn > 1e-13 * amax) || j + 1 == d) break;
        beta.push_back(bn);
    }
    beta.resize(alpha.size(), 0.0);
    tridiag_extremes(alpha, beta, &out[0], &out[1]);
    out[2] = fro2_known > 0.0 ? fro2_known : fro2;
    return RK_OK;
}

}  // namespace rk
