// rk_adjoint.cu -- differentiation form: the adjoint of x = argmin ||A x - b||
// (Eq. (ls_system)) for a loss L(x).  Differentiating the normal equations
// A^T A x = A^T b gives A^T A dx = dA^T r - A^T dA x + A^T db with r = b - A x, so
// with g = (A^T A)^{-1} dL/dx and y = A g:
//   dL = < r g^T - y x^T, dA > + < y, db >,   grad_b = y,   grad_A = r g^T - y x^T.
// y is the minimum-norm solution of A^T y = dL/dx, which Kaczmarz reaches from
// y = 0 (Section 2.1: on underdetermined systems Kaczmarz converges to the
// least Euclidean norm solution); it is computed by RKAB on the rows of A^T (a
// transposed copy of A), and g by RKAB on the consistent system A g = y.
#include <cstdint>

#include "rk_common.cuh"
#include "rk_internal.h"

namespace rk {

// At[j][i] = A[i][j] through 32 x 32 shared-memory tiles (coalesced both ways).
__global__ void __launch_bounds__(256) transpose_kernel(const float* __restrict__ A, int64_t m, int64_t n,
                                                        int64_t lda, float* __restrict__ At, int64_t ldt) {
    __shared__ float tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, j = j0 + tx;
        tile[r][tx] = (i < m && j < n) ? __ldg(A + i * lda + j) : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r, i = i0 + tx;
        if (j < n && i < m) At[j * ldt + i] = tile[tx][r];
    }
}

// G[i][j] = r_i g_j - y_i x_j (the rank-2 gradient of A), float4 stores along j.
// One CTA covers one row chunk; g and x are read once per CTA tile from L2.
__global__ void __launch_bounds__(256) rank2_kernel(const float* __restrict__ r, const float* __restrict__ g,
                                                    const float* __restrict__ y, const float* __restrict__ x,
                                                    int64_t m, int64_t n, float* __restrict__ G, int64_t ldg) {
    const int64_t n4 = n >> 2;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const float ri = __ldg(r + i), yi = __ldg(y + i);
        float* Gi = G + i * ldg;
        for (int64_t c = threadIdx.x; c < n4; c += blockDim.x) {
            const int64_t j = c * 4;
            float4 o;
            o.x = fmaf(ri, __ldg(g + j), -yi * __ldg(x + j));
            o.y = fmaf(ri, __ldg(g + j + 1), -yi * __ldg(x + j + 1));
            o.z = fmaf(ri, __ldg(g + j + 2), -yi * __ldg(x + j + 2));
            o.w = fmaf(ri, __ldg(g + j + 3), -yi * __ldg(x + j + 3));
            __stcs(reinterpret_cast<float4*>(Gi + j), o);
        }
        for (int64_t j = n4 * 4 + threadIdx.x; j < n; j += blockDim.x)
            Gi[j] = fmaf(ri, __ldg(g + j), -yi * __ldg(x + j));
    }
}

__global__ void narrow64_kernel(float* __restrict__ o, const double* __restrict__ v, int64_t m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)v[i];
}

static int grid_cap(int64_t want) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = (int64_t)sms * 16;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

int launch_transpose(const float* A, int64_t m, int64_t n, int64_t lda, float* At, int64_t ldt,
                     cudaStream_t st) {
    const int64_t gx = (n + 31) / 32, gy = (m + 31) / 32;
    if (gy > 65535) return RK_EINVAL;
    transpose_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(A, m, n, lda, At, ldt);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

int launch_rank2(const float* r, const float* g, const float* y, const float* x, int64_t m, int64_t n,
                 float* G, int64_t ldg, cudaStream_t st) {
    rank2_kernel<<<grid_cap(m), 256, 0, st>>>(r, g, y, x, m, n, G, ldg);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

// Workspace: r64 (m doubles) | r32 (m floats) | zeros (max(m, n) floats) |
//            solve workspace for A^T (q_t) | solve workspace for A (q) | residual workspace
size_t adjoint_ws_bytes(const Plan* pa, const Plan* pt, int q_t, int q) {
    const int64_t m = pa->m, n = pa->n;
    const int64_t zn = (m > n ? m : n) + 4;
    return align256((size_t)m * 8) + align256((size_t)m * 4) + align256((size_t)zn * 4) +
           align256(solve_ws_bytes(pt, q_t)) + align256(solve_ws_bytes(pa, q)) +
           align256(residual_ws_bytes(m, n));
}

int run_adjoint(const Plan* pa, const Plan* pt, const float* b, const float* x, const float* gx,
                int q_t, int q, int64_t alpha_t, int64_t rounds_t, int64_t alpha, int64_t rounds, uint64_t seed,
                const rk_opts& ot, const rk_opts& oa, float* grad_b, float* grad_A, int64_t ldg,
                float* g_out, void* ws, cudaStream_t st) {
    const int64_t m = pa->m, n = pa->n;
    uint8_t* p = static_cast<uint8_t*>(ws);
    double* r64 = reinterpret_cast<double*>(p);
    p += align256((size_t)m * 8);
    float* r32 = reinterpret_cast<float*>(p);
    p += align256((size_t)m * 4);
    float* zeros = reinterpret_cast<float*>(p);
    const int64_t zn = (m > n ? m : n) + 4;
    p += align256((size_t)zn * 4);
    void* wt = p;
    p += align256(solve_ws_bytes(pt, q_t));
    void* wa = p;
    p += align256(solve_ws_bytes(pa, q));
    void* wr = p;
    if (cudaMemsetAsync(zeros, 0, (size_t)zn * 4, st) != cudaSuccess) return RK_ECUDA;

    // (1) y: minimum-norm solution of A^T y = gx from y = 0 (Philox stream id 1) -> grad_b
    SolveArgs s1;
    s1.plan = pt;
    s1.b = gx;
    s1.x0 = zeros;
    s1.x = grad_b;
    s1.q = q_t;
    s1.alpha = alpha_t;
    s1.rounds = rounds_t;
    s1.seed = seed;
    s1.opts = ot;
    s1.opts.stream_id = 1u;
    s1.opts.round0 = 0;
    s1.info = static_cast<SolveInfo*>(wt);
    s1.ldv = (pt->n + 3) / 4 * 4;
    s1.V = reinterpret_cast<float*>(static_cast<uint8_t*>(wt) + align256(sizeof(SolveInfo)));
    if (cudaMemsetAsync(s1.info, 0, sizeof(SolveInfo), st) != cudaSuccess) return RK_ECUDA;
    int rc = launch_solve(s1, st);
    if (rc != RK_OK) return rc;
    // (2) g: A g = y from g = 0 (stream id 2)
    float* g_buf = g_out;
    SolveArgs s2 = s1;
    s2.plan = pa;
    s2.b = grad_b;
    s2.x0 = zeros;
    s2.x = g_buf;
    s2.q = q;
    s2.alpha = alpha;
    s2.rounds = rounds;
    s2.opts = oa;
    s2.opts.stream_id = 2u;
    s2.opts.round0 = 0;
    s2.info = static_cast<SolveInfo*>(wa);
    s2.ldv = (pa->n + 3) / 4 * 4;
    s2.V = reinterpret_cast<float*>(static_cast<uint8_t*>(wa) + align256(sizeof(SolveInfo)));
    if (cudaMemsetAsync(s2.info, 0, sizeof(SolveInfo), st) != cudaSuccess) return RK_ECUDA;
    rc = launch_solve(s2, st);
    if (rc != RK_OK) return rc;
    // (3) r = b - A x with float64 accumulation, rounded to float32
    rc = launch_residual(static_cast<const float*>(pa->A), m, n, pa->lda, b, x, r64, nullptr, 0, wr, st);
    if (rc != RK_OK) return rc;
    narrow64_kernel<<<grid_cap((m + 255) / 256), 256, 0, st>>>(r32, r64, m);
    count_launch();
    // (4) grad_A = r g^T - y x^T
    rc = launch_rank2(r32, g_buf, grad_b, x, m, n, grad_A, ldg, st);
    if (rc != RK_OK) return rc;
    // device status of both solves
    SolveInfo i1, i2;
    if (cudaMemcpyAsync(&i1, s1.info, sizeof(i1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&i2, s2.info, sizeof(i2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RK_ECUDA;
    if (i1.status != 0) return i1.status;
    if (i2.status != 0) return i2.status;
    return RK_OK;
}

}  // namespace rk
