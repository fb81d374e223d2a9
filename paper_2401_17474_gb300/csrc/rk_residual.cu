// rk_residual.cu -- residual of Eq. (system) / Eq. (ls_system) with float32 A
// and FP64-class accumulation: r = b - A x, ||r||_2 and the normal-equation
// residual ||A^T r||_2.  All reductions run in a fixed order (warp butterfly,
// then block partials summed in ascending block order), so results are the
// same on every run.
#include <cstdint>

#include "rk_common.cuh"
#include "rk_internal.h"

namespace rk {

constexpr int kResThreads = 256;
constexpr int kAtrCols = 1024;  // columns per CTA of the A^T r pass (one float4 per thread)

struct ResWs {
    double* r;         // m (used when the caller passes no r)
    float2* rs;        // m: r_i split into float32 (hi, lo) for the A^T r pass
    double* rr_part;   // per-block sums of r_i^2
    double* atr_part;  // [row chunks][n]
    double* atr_bpart; // per-block sums of c_j^2 for ||A^T r||
    double* norms;     // [2] when the caller passes none
};

static int res_blocks(int64_t m) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (m + (kResThreads / 32) - 1) / (kResThreads / 32);
    const int64_t cap = (int64_t)sms * 8;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

static int atr_chunks(int64_t m, int64_t n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ctiles = (n + kAtrCols - 1) / kAtrCols;
    int64_t chunks = ((int64_t)sms * 4 + ctiles - 1) / ctiles;
    if (chunks > m) chunks = m;
    return (int)(chunks < 1 ? 1 : chunks);
}

// Exact product and compensated (TwoSum) accumulation in a pair of float32:
// a x = p + e exactly (e = fma(a, x, -p)); (hi, lo) += p + e with the rounding
// error of hi + p recovered by TwoSum (Knuth).  Over k terms the pair's error is
// about 2^-46 sum|a_j x_j| (the float32 pair carries ~48 significant bits), which
// is tighter than float64 recursive summation (k 2^-53 sum|a_j x_j|) once k > 2^7;
// the pairs of the 32 lanes are then added in float64.
// The _rn intrinsics are never contracted into fused multiply-adds, which the
// error terms rely on.
__device__ __forceinline__ void df_acc(float& hi, float& lo, float a, float x) {
    const float p = __fmul_rn(a, x);
    const float e = fmaf(a, x, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// One warp per row: r_i = b_i - sum_j a_ij x_j with FP64-class accumulation
// (compensated float32 pairs per lane, float64 across lanes) -- the float64 pipe
// of the device is not needed per element, so the pass runs at memory speed.
__global__ void __launch_bounds__(kResThreads) residual_rows_kernel(
    const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, const float* __restrict__ b,
    const float* __restrict__ x, double* __restrict__ r, float2* __restrict__ rs,
    double* __restrict__ rr_part) {
    __shared__ double s_rr[kResThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n4 = n >> 2;
    // x as float4 when it is 16-byte aligned (the rows always are)
    const float4* x4 = ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) ? reinterpret_cast<const float4*>(x) : nullptr;
    double rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * (kResThreads / 32) + warp; i < m;
         i += (int64_t)gridDim.x * (kResThreads / 32)) {
        const float* a = A + i * lda;
        const float4* a4 = reinterpret_cast<const float4*>(a);
        float hi = 0.f, lo = 0.f;
        int64_t c = lane;
        if (x4) {
            // four float4 of the row in flight per lane (streamed once: evict first)
            for (; c + 96 < n4; c += 128) {
                float4 v[4], xv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v[u] = __ldcs(a4 + c + 32 * u);
                    xv[u] = __ldg(x4 + c + 32 * u);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    df_acc(hi, lo, v[u].x, xv[u].x);
                    df_acc(hi, lo, v[u].y, xv[u].y);
                    df_acc(hi, lo, v[u].z, xv[u].z);
                    df_acc(hi, lo, v[u].w, xv[u].w);
                }
            }
        }
        for (; c < n4; c += 32) {
            const float4 v = __ldcs(a4 + c);
            const int64_t j = c * 4;
            df_acc(hi, lo, v.x, __ldg(x + j));
            df_acc(hi, lo, v.y, __ldg(x + j + 1));
            df_acc(hi, lo, v.z, __ldg(x + j + 2));
            df_acc(hi, lo, v.w, __ldg(x + j + 3));
        }
        for (int64_t j = n4 * 4 + lane; j < n; j += 32) df_acc(hi, lo, __ldg(a + j), __ldg(x + j));
        double acc = (double)hi + (double)lo;
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double ri = (b ? (double)__ldg(b + i) : 0.0) - acc;   // no b: r = -A x
        if (lane == 0) {
            r[i] = ri;
            const float rh = (float)ri;
            rs[i] = make_float2(rh, (float)(ri - (double)rh));
            rr = fma(ri, ri, rr);
        }
    }
    if (lane == 0) s_rr[warp] = rr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kResThreads / 32; ++w) s += s_rr[w];
        rr_part[blockIdx.x] = s;
    }
}

// (hi, lo) += a (rh + rl) for a float32 a and a float64 r split into float32
// rh = fl(r), rl = fl(r - rh): a rh = p + e exactly, a rl is kept rounded (its
// error is below 2^-48 |a r|), and the sum goes through TwoSum as in df_acc.
__device__ __forceinline__ void df_acc_split(float& hi, float& lo, float a, float rh, float rl) {
    const float p = __fmul_rn(a, rh);
    const float e = fmaf(a, rh, -p);
    const float t = fmaf(a, rl, e);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, t));
}

// CTA (column tile, row chunk): partial (A^T r)_j over the chunk's rows, one
// float4 of columns per thread, accumulated in compensated float32 pairs (about
// 2^-46 relative to sum_i |a_ij r_i|) and written as float64.
__global__ void __launch_bounds__(kResThreads) residual_atr_kernel(
    const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, const float2* __restrict__ rs,
    int chunks, double* __restrict__ atr_part) {
    const int64_t ctile = blockIdx.x;
    const int chunk = blockIdx.y;
    const int64_t rows_per = (m + chunks - 1) / chunks;
    const int64_t i0 = (int64_t)chunk * rows_per;
    const int64_t i1 = min(m, i0 + rows_per);
    const int64_t j0 = ctile * kAtrCols + (int64_t)threadIdx.x * 4;
    if (j0 >= n) return;
    float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f;
    const bool full4 = (j0 + 3 < n);
    int64_t i = i0;
    if (full4) {
        // four rows in flight per thread; rows in ascending order as below
        for (; i + 4 <= i1; i += 4) {
            float4 v[4];
            float2 rr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = __ldcs(reinterpret_cast<const float4*>(A + (i + u) * lda + j0));
                rr[u] = __ldg(rs + i + u);   // r_i = rh + rl, split once per row
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                df_acc_split(h0, l0, v[u].x, rr[u].x, rr[u].y);
                df_acc_split(h1, l1, v[u].y, rr[u].x, rr[u].y);
                df_acc_split(h2, l2, v[u].z, rr[u].x, rr[u].y);
                df_acc_split(h3, l3, v[u].w, rr[u].x, rr[u].y);
            }
        }
    }
    for (; i < i1; ++i) {
        const float2 rr = __ldg(rs + i);
        const float rh = rr.x, rl = rr.y;
        const float* a = A + i * lda + j0;
        if (full4) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(a));
            df_acc_split(h0, l0, v.x, rh, rl);
            df_acc_split(h1, l1, v.y, rh, rl);
            df_acc_split(h2, l2, v.z, rh, rl);
            df_acc_split(h3, l3, v.w, rh, rl);
        } else {
            df_acc_split(h0, l0, __ldg(a), rh, rl);
            if (j0 + 1 < n) df_acc_split(h1, l1, __ldg(a + 1), rh, rl);
            if (j0 + 2 < n) df_acc_split(h2, l2, __ldg(a + 2), rh, rl);
        }
    }
    double* out = atr_part + (size_t)chunk * (size_t)n + j0;
    out[0] = (double)h0 + (double)l0;
    if (j0 + 1 < n) out[1] = (double)h1 + (double)l1;
    if (j0 + 2 < n) out[2] = (double)h2 + (double)l2;
    if (j0 + 3 < n) out[3] = (double)h3 + (double)l3;
}

// Columns of A^T r over the grid: c_j = sum of the chunk partials of column j (chunks
// in ascending order), and per block the sum of c_j^2 over its columns (a fixed tree).
__global__ void __launch_bounds__(kResThreads) atr_norm_parts_kernel(const double* __restrict__ atr_part,
                                                                     int chunks, int64_t n,
                                                                     double* __restrict__ bpart) {
    __shared__ double s_part[kResThreads];
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * kResThreads + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * kResThreads) {
        double c = 0.0;
        for (int k = 0; k < chunks; ++k) c += atr_part[(size_t)k * (size_t)n + j];
        acc = fma(c, c, acc);
    }
    s_part[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kResThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s_part[threadIdx.x] += s_part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) bpart[blockIdx.x] = s_part[0];
}

static int atr_norm_blocks(int64_t n) {
    const int64_t g = (n + kResThreads - 1) / kResThreads;
    return (int)(g < 512 ? g : 512);
}

// One thread: norms[0] = sqrt(sum of rr partials), norms[1] = ||A^T r|| from the block
// partials of atr_norm_parts_kernel (both summed in block order).
__global__ void residual_finish_kernel(const double* __restrict__ rr_part, int nblocks,
                                       const double* __restrict__ atr_bpart, int nbp,
                                       double* __restrict__ norms) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < nblocks; ++k) s += rr_part[k];
    norms[0] = sqrt(s);
    if (!atr_bpart) return;
    double t = 0.0;
    for (int k = 0; k < nbp; ++k) t += atr_bpart[k];
    norms[1] = sqrt(t);
}

static ResWs carve(void* base, int64_t m, int64_t n) {
    uint8_t* p = static_cast<uint8_t*>(base);
    ResWs w;
    w.norms = reinterpret_cast<double*>(p);
    p += 256;
    w.r = reinterpret_cast<double*>(p);
    p += align256((size_t)m * 8);
    w.rs = reinterpret_cast<float2*>(p);
    p += align256((size_t)m * 8);
    w.rr_part = reinterpret_cast<double*>(p);
    p += align256((size_t)res_blocks(m) * 8);
    w.atr_part = reinterpret_cast<double*>(p);
    p += align256((size_t)atr_chunks(m, n) * (size_t)n * 8);
    w.atr_bpart = reinterpret_cast<double*>(p);
    return w;
}

size_t residual_ws_bytes(int64_t m, int64_t n) {
    return 256 + 2 * align256((size_t)m * 8) + align256((size_t)res_blocks(m) * 8) +
           align256((size_t)atr_chunks(m, n) * (size_t)n * 8) + align256((size_t)atr_norm_blocks(n) * 8);
}

int launch_residual(const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
                    const float* x, double* r, double* norms_out, int want_atr, void* ws,
                    cudaStream_t st) {
    ResWs w = carve(ws, m, n);
    double* rv = r ? r : w.r;
    double* norms = norms_out ? norms_out : w.norms;
    const int nb = res_blocks(m);
    residual_rows_kernel<<<nb, kResThreads, 0, st>>>(A, m, n, lda, b, x, rv, w.rs, w.rr_part);
    count_launch();
    int chunks = 0;
    if (want_atr) {
        chunks = atr_chunks(m, n);
        dim3 grid((unsigned)((n + kAtrCols - 1) / kAtrCols), (unsigned)chunks);
        residual_atr_kernel<<<grid, kResThreads, 0, st>>>(A, m, n, lda, w.rs, chunks, w.atr_part);
        count_launch();
    }
    const int nbp = atr_norm_blocks(n);
    if (want_atr) {
        atr_norm_parts_kernel<<<nbp, kResThreads, 0, st>>>(w.atr_part, chunks, n, w.atr_bpart);
        count_launch();
    }
    residual_finish_kernel<<<1, 32, 0, st>>>(w.rr_part, nb, want_atr ? w.atr_bpart : nullptr, nbp, norms);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

// w_j = -sum_c part[c][j] (chunks in ascending order): with r = -A v this is A^T A v.
__global__ void __launch_bounds__(kResThreads) gather_neg_kernel(const double* __restrict__ part,
                                                                  int chunks, int64_t n,
                                                                  double* __restrict__ w) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double c = 0.0;
        for (int k = 0; k < chunks; ++k) c += part[(size_t)k * (size_t)n + j];
        w[j] = -c;
    }
}

// w = A^T A v for float32 A and v: r = -A v by the row kernel (no right-hand side),
// then the A^T r pass and the fixed-order sum of its row-chunk partials.  Two
// passes over A; the workspace is that of launch_residual.
int launch_normal_matvec(const float* A, int64_t m, int64_t n, int64_t lda, const float* v,
                         double* w, void* ws, cudaStream_t st) {
    ResWs rw = carve(ws, m, n);
    const int nb = res_blocks(m);
    residual_rows_kernel<<<nb, kResThreads, 0, st>>>(A, m, n, lda, nullptr, v, rw.r, rw.rs, rw.rr_part);
    count_launch();
    const int chunks = atr_chunks(m, n);
    dim3 grid((unsigned)((n + kAtrCols - 1) / kAtrCols), (unsigned)chunks);
    residual_atr_kernel<<<grid, kResThreads, 0, st>>>(A, m, n, lda, rw.rs, chunks, rw.atr_part);
    count_launch();
    const int64_t gb = (n + kResThreads - 1) / kResThreads;
    gather_neg_kernel<<<(unsigned)(gb < 1024 ? gb : 1024), kResThreads, 0, st>>>(rw.atr_part, chunks, n, w);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

// r = -A v for float32 A and v (the row pass of the residual without a right-hand
// side), written to r (m doubles).  One pass over A.
int launch_rows_matvec(const float* A, int64_t m, int64_t n, int64_t lda, const float* v, double* r,
                       void* ws, cudaStream_t st) {
    ResWs rw = carve(ws, m, n);
    residual_rows_kernel<<<res_blocks(m), kResThreads, 0, st>>>(A, m, n, lda, nullptr, v, r, rw.rs,
                                                                rw.rr_part);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

// rs_i = u_i split into float32 (hi, lo), the input format of the A^T r pass.
__global__ void split_rows_kernel(const double* __restrict__ u, int64_t m, float2* __restrict__ rs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)u[i];
        rs[i] = make_float2(h, (float)(u[i] - (double)h));
    }
}

// w = -A^T u for float32 A and float64 u (m entries): the A^T r pass of the residual
// with r = u, then the fixed-order sum of its row-chunk partials.  One pass over A;
// u may share storage with w (u is consumed before w is written).
int launch_transpose_matvec(const float* A, int64_t m, int64_t n, int64_t lda, const double* u,
                            double* w, void* ws, cudaStream_t st) {
    ResWs rw = carve(ws, m, n);
    const int64_t gs = (m + kResThreads - 1) / kResThreads;
    split_rows_kernel<<<(unsigned)(gs < 2048 ? gs : 2048), kResThreads, 0, st>>>(u, m, rw.rs);
    count_launch();
    const int chunks = atr_chunks(m, n);
    dim3 grid((unsigned)((n + kAtrCols - 1) / kAtrCols), (unsigned)chunks);
    residual_atr_kernel<<<grid, kResThreads, 0, st>>>(A, m, n, lda, rw.rs, chunks, rw.atr_part);
    count_launch();
    const int64_t gb = (n + kResThreads - 1) / kResThreads;
    gather_neg_kernel<<<(unsigned)(gb < 1024 ? gb : 1024), kResThreads, 0, st>>>(rw.atr_part, chunks, n, w);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

}  // namespace rk
