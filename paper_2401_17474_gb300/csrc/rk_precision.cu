// rk_precision.cu -- precision form of the solve: stored-row quantisers
// (float32 -> bfloat16 round-to-nearest-even; float32 -> FP8 e4m3 with a
// per-row float32 scale amax_i / 448, round-to-nearest-even, saturating), and
// outer iterative refinement: r = b - A x with the float32 master A and float64
// accumulation, the correction d from an RKAB solve of A~ d = r on the stored
// copy A~ starting at d = 0, then x <- x + d.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cmath>
#include <cstdint>

#include "rk_common.cuh"
#include "rk_internal.h"

namespace rk {

constexpr int kQThreads = 256;

// One CTA per row (grid-stride over rows): out[i][j] = bf16_rn(A[i][j]), zero padding.
__global__ void __launch_bounds__(kQThreads) quant_bf16_kernel(const float* __restrict__ A, int64_t m,
                                                               int64_t n, int64_t lda,
                                                               uint16_t* __restrict__ out, int64_t ldo) {
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const float* a = A + i * lda;
        uint16_t* o = out + i * ldo;
        for (int64_t j = threadIdx.x; j < ldo; j += blockDim.x) {
            o[j] = j < n ? __bfloat16_as_ushort(__float2bfloat16_rn(__ldg(a + j))) : (uint16_t)0;
        }
    }
}

// One CTA per row: s_i = amax_i / 448 (1 for an all-zero row), out = e4m3_satfinite(a / s_i).
__global__ void __launch_bounds__(kQThreads) quant_fp8_kernel(const float* __restrict__ A, int64_t m,
                                                              int64_t n, int64_t lda,
                                                              uint8_t* __restrict__ out, int64_t ldo,
                                                              float* __restrict__ scale) {
    __shared__ float s_max[kQThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const float* a = A + i * lda;
        float mx = 0.f;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(__ldg(a + j)));
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_max[warp] = mx;
        __syncthreads();
        mx = 0.f;
        for (int w = 0; w < kQThreads / 32; ++w) mx = fmaxf(mx, s_max[w]);
        const float s = mx > 0.f ? __fdiv_rn(mx, 448.0f) : 1.0f;
        if (threadIdx.x == 0) scale[i] = s;
        uint8_t* o = out + i * ldo;
        for (int64_t j = threadIdx.x; j < ldo; j += blockDim.x) {
            o[j] = j < n ? (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(__ldg(a + j), s), __NV_SATFINITE, __NV_E4M3)
                         : (uint8_t)0;
        }
        __syncthreads();
    }
}

// x <- x + d (float32)
__global__ void axpy_kernel(float* __restrict__ x, const float* __restrict__ d, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        x[j] += d[j];
}

// r32 <- float32(r64)
__global__ void narrow_kernel(float* __restrict__ r32, const double* __restrict__ r64, int64_t m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        r32[i] = (float)r64[i];
}

// out[0] = ||x - xr||^2, out[1] = ||xr||^2 (float64, one block, fixed order).
__global__ void __launch_bounds__(kQThreads) relerr_kernel(const float* __restrict__ x,
                                                           const float* __restrict__ xr, int64_t n,
                                                           double* out) {
    __shared__ double s_e[kQThreads], s_r[kQThreads];
    double e = 0.0, r = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += kQThreads) {
        const double dd = (double)x[j] - (double)xr[j];
        e = fma(dd, dd, e);
        r = fma((double)xr[j], (double)xr[j], r);
    }
    s_e[threadIdx.x] = e;
    s_r[threadIdx.x] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double E = 0.0, R = 0.0;
        for (int k = 0; k < kQThreads; ++k) {
            E += s_e[k];
            R += s_r[k];
        }
        out[0] = E;
        out[1] = R;
    }
}

static int qgrid(int64_t m) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = (int64_t)sms * 8;
    return (int)(m < cap ? m : cap);
}

int launch_quantize(const float* A, int64_t m, int64_t n, int64_t lda, rk_dtype dt, void* out,
                    int64_t ldo, float* row_scale, cudaStream_t st) {
    if (dt == RK_BF16) {
        quant_bf16_kernel<<<qgrid(m), kQThreads, 0, st>>>(A, m, n, lda, static_cast<uint16_t*>(out), ldo);
    } else if (dt == RK_FP8E4M3) {
        quant_fp8_kernel<<<qgrid(m), kQThreads, 0, st>>>(A, m, n, lda, static_cast<uint8_t*>(out), ldo,
                                                         row_scale);
    } else {
        return RK_EINVAL;
    }
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

// Refinement workspace: [256 B header: 2 doubles of the error norms]
//   r64 (m doubles) | r32 (m floats) | d (n4*4 floats) | zero (n4*4 floats)
//   | residual workspace | solve workspace (q)
struct RefineWs {
    double* err;
    double* r64;
    float* r32;
    float* d;
    float* zero;
    float* cref;   // x_ref - x: the correction that meets the criterion exactly
    void* res_ws;
    size_t res_bytes;
    void* solve_ws;
    size_t solve_bytes;
};

static RefineWs refine_carve(void* base, const Plan* pl, int q) {
    uint8_t* p = static_cast<uint8_t*>(base);
    const size_t ldv = (size_t)((pl->n + 3) / 4) * 4;
    RefineWs w;
    w.err = reinterpret_cast<double*>(p);
    p += 256;
    w.r64 = reinterpret_cast<double*>(p);
    p += align256((size_t)pl->m * 8);
    w.r32 = reinterpret_cast<float*>(p);
    p += align256((size_t)pl->m * 4);
    w.d = reinterpret_cast<float*>(p);
    p += align256(ldv * 4);
    w.zero = reinterpret_cast<float*>(p);
    p += align256(ldv * 4);
    w.cref = reinterpret_cast<float*>(p);
    p += align256(ldv * 4);
    w.res_ws = p;
    w.res_bytes = align256(residual_ws_bytes(pl->m, pl->n));
    p += w.res_bytes;
    w.solve_ws = p;
    w.solve_bytes = solve_ws_bytes(pl, q);
    return w;
}

size_t refine_ws_bytes(const Plan* pl, int q) {
    const size_t ldv = (size_t)((pl->n + 3) / 4) * 4;
    return 256 + align256((size_t)pl->m * 8) + align256((size_t)pl->m * 4) + 3 * align256(ldv * 4) +
           align256(residual_ws_bytes(pl->m, pl->n)) + solve_ws_bytes(pl, q);
}

// c = x_ref - x (float32)
__global__ void sub_kernel(const float* __restrict__ xr, const float* __restrict__ x, int64_t n,
                           float* __restrict__ c) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        c[j] = xr[j] - x[j];
}

int run_refine(const Plan* lowp, const float* A32, int64_t lda32, const float* b, const float* x0,
               float* x, int q, int64_t alpha, int64_t inner_rounds, int64_t max_outer,
               uint64_t seed, const rk_opts& o, void* ws, cudaStream_t st, int64_t* outer_done,
               double* last_metric) {
    const int64_t m = lowp->m, n = lowp->n;
    RefineWs w = refine_carve(ws, lowp, q);
    if (outer_done) *outer_done = 0;
    if (last_metric) *last_metric = -1.0;
    if (x != x0 && cudaMemcpyAsync(x, x0, (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RK_ECUDA;
    if (cudaMemsetAsync(w.zero, 0, (size_t)n * 4, st) != cudaSuccess) return RK_ECUDA;
    const int g = qgrid((m + 255) / 256 + 1);
    const int gn = qgrid((n + 255) / 256 + 1);
    // with a reference solution and a tolerance, every inner solve also stops as soon as
    // x + d meets the criterion: its reference is c = x_ref - x and its tolerance
    // tol ||x_ref|| / ||c|| (||x + d - x_ref|| = ||d - c||); err0 holds ||x - x_ref||^2 and
    // ||x_ref||^2 of the current x
    const bool exact_stop = o.criterion == 1 && o.x_ref && o.tol > 0.0;
    double err0[2] = {0.0, 0.0};
    if (exact_stop) {
        relerr_kernel<<<1, kQThreads, 0, st>>>(x, o.x_ref, n, w.err);
        count_launch();
        if (cudaMemcpyAsync(err0, w.err, sizeof(err0), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RK_ECUDA;
    }
    for (int64_t outer = 0; outer < max_outer; ++outer) {
        int rc = launch_residual(A32, m, n, lda32, b, x, w.r64, nullptr, 0, w.res_ws, st);
        if (rc != RK_OK) return rc;
        narrow_kernel<<<g, 256, 0, st>>>(w.r32, w.r64, m);
        count_launch();
        SolveArgs a;
        a.plan = lowp;
        a.b = w.r32;
        a.x0 = w.zero;
        a.x = w.d;
        a.q = q;
        a.alpha = alpha;
        a.rounds = inner_rounds;
        a.seed = seed;
        rk_opts io;
        rk_opts_default(&io);
        io.omega = o.omega;
        io.check_every = 0;
        io.stream_id = 3u + ((uint32_t)outer << 8);
        io.timeout_s = o.timeout_s;
        io.lookahead = o.lookahead;
        io.sampling = o.sampling;
        io.row_weight = o.row_weight;
        io.worker_weight = o.worker_weight;
        if (exact_stop && err0[0] > 0.0) {
            sub_kernel<<<gn, 256, 0, st>>>(o.x_ref, x, n, w.cref);
            count_launch();
            io.criterion = 1;
            io.x_ref = w.cref;
            io.check_every = 1;
            io.tol = o.tol * std::sqrt(err0[1] / err0[0]);
        }
        a.opts = io;
        a.info = static_cast<SolveInfo*>(w.solve_ws);
        a.ldv = (n + 3) / 4 * 4;
        a.V = reinterpret_cast<float*>(static_cast<uint8_t*>(w.solve_ws) + align256(sizeof(SolveInfo)));
        if (cudaMemsetAsync(a.info, 0, sizeof(SolveInfo), st) != cudaSuccess) return RK_ECUDA;
        rc = launch_solve(a, st);
        if (rc != RK_OK) return rc;
        axpy_kernel<<<qgrid((n + 255) / 256 + 1), 256, 0, st>>>(x, w.d, n);
        count_launch();
        SolveInfo info;
        if (cudaMemcpyAsync(&info, a.info, sizeof(info), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return RK_ECUDA;
        double err[2] = {0.0, 0.0};
        if (o.criterion == 1) {
            relerr_kernel<<<1, kQThreads, 0, st>>>(x, o.x_ref, n, w.err);
            count_launch();
            if (cudaMemcpyAsync(err, w.err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess)
                return RK_ECUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return RK_ECUDA;
        if (info.status != 0) return info.status;
        if (outer_done) *outer_done = outer + 1;
        if (o.criterion == 1) {
            const double metric = err[1] > 0.0 ? std::sqrt(err[0] / err[1]) : std::sqrt(err[0]);
            if (last_metric) *last_metric = metric;
            if (!std::isfinite(metric)) return RK_EDIVERGED;
            if (o.tol > 0.0 && metric < o.tol) break;
            err0[0] = err[0];
            err0[1] = err[1];
        }
    }
    return RK_OK;
}

}  // namespace rk
