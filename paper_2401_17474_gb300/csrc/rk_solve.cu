// rk_solve.cu -- host side of the persistent RKAB solve (kernel in
// rk_solve_kernel.cuh): choice of the CTA shape for n, shared-memory stage
// count, cooperative launch; and the row-draw test kernel.
#include <algorithm>
#include <cstdint>

#include "rk_cluster_kernel.cuh"
#include "rk_solve_kernel.cuh"

namespace rk {

static size_t elem_size(rk_dtype dt) { return dt == RK_F32 ? 4 : (dt == RK_BF16 ? 2 : 1); }

__global__ void sample_indices_kernel(const uint64_t* __restrict__ thr64,
                                      const uint32_t* __restrict__ alias, uint64_t m,
                                      uint64_t seed, uint32_t worker, uint32_t stream_id,
                                      uint64_t t0, int64_t count, uint32_t* out,
                                      const SetupInfo* setup) {
    if (setup->status != 0) return;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        out[k] = sample_row(seed, worker, stream_id, t0 + (uint64_t)k, m, thr64, alias);
    }
}

// Consumer threads per CTA: few warps keep the per-projection reduction short,
// enough slices per thread keep the FMA pipe busy, and the register file bounds
// x, d and the row slices (256 consumers + 1 producer warp may use 168
// registers/thread, 512 + 1 only 96): 32 threads up to n = 512, 128 up to
// n = 2560, 256 up to n = 16384 (beyond 10240 columns with the row re-read from
// shared memory: half the warps of a 512-thread CTA to reduce each dot over), else
// 512; then the smallest instantiated slices-per-thread count that covers n.
static const SolveVariant* find_variant(const SolveVariant* tab, int count, int nt, int n4, int w,
                                        int minb, bool jac, bool xs = false) {
    const int need = (n4 + nt - 1) / nt;
    const SolveVariant* best = nullptr;
    for (int i = 0; i < count; ++i) {
        if (tab[i].minb == minb && tab[i].jac == jac && tab[i].xs == xs && tab[i].nt == nt && tab[i].w == w &&
            tab[i].vpt >= need && (!best || tab[i].vpt < best->vpt))
            best = &tab[i];
    }
    return best;
}

// Stored types whose rows of 10K-16K columns run the variant with x in shared memory
// (bit 1 << dtype): FP8 rows, whose decoding makes the consumers the bound, gain from
// the single pass over each row with the decoded row kept in registers (measured at
// 100000 x 16000, q = 132: 12.7 against 16.1 ms a round); BF16 rows (13.3 against
// 13.1 ms) and float32 rows (18.9 against 18.2 ms) do not.
#ifndef RK_SOLVE_XS_DTYPES
#define RK_SOLVE_XS_DTYPES 4
#endif


static const SolveVariant* pick_variant(rk_dtype dt, int n4, int w, int minb = 1, bool jac = false) {
    int count = 0;
    const SolveVariant* tab = dt == RK_F32 ? solve_variants_f32(&count)
                            : dt == RK_BF16 ? solve_variants_bf16(&count)
                                            : solve_variants_fp8(&count);
    int nt = n4 <= 32 * 4 ? 32 : (n4 <= 128 * 5 ? 128 : (n4 <= 256 * 10 ? 256 : 512));
    // two workers per SM: 128 or 256 consumers, slices re-read from shared memory
    if (minb == 2) nt = n4 <= 128 * 5 ? 128 : 256;
    if (nt == 512 && n4 <= 256 * 16) {
        if (w == 1 && minb == 1 && !jac && ((RK_SOLVE_XS_DTYPES >> (int)dt) & 1)) {
            const SolveVariant* v = find_variant(tab, count, 256, n4, w, minb, jac, true);
            if (v) return v;
        }
        const SolveVariant* v = find_variant(tab, count, 256, n4, w, minb, jac);
        if (v) return v;
    }
    return find_variant(tab, count, nt, n4, w, minb, jac);
}

static const int kMaxStages = 16;

// Shared memory of a variant's x (NT * VPT float4) when it keeps x there.
static size_t xs_bytes(const SolveVariant* v) { return v->xs ? (size_t)v->nt * v->vpt * 16 : 0; }

static int stages_for(uint32_t stride, int nt, int smem_max) {
    int S = 0;
    while (S < kMaxStages &&
           (size_t)(S + 1) * stride + solve_ctrl_bytes(S + 1, nt) <= (size_t)smem_max)
        ++S;
    return S;
}

int launch_colsplit_solve(const SolveArgs& a, const KParams& base, cudaStream_t st, int smem_max, int sms);

// Cluster path: each worker is a cluster of C CTAs splitting the row's columns.
static int launch_cluster_solve(const SolveArgs& a, const KParams& base, int C, cudaStream_t st,
                                int smem_max) {
    const Plan* pl = a.plan;
    const int n4 = base.n4;
    const uint32_t eb = (uint32_t)elem_size(pl->dt);
    const int chunk = ((n4 + C - 1) / C + 3) / 4 * 4;
    if ((C - 1) * chunk >= n4) return RK_EINVAL;   // every CTA must own part of the row
    int count = 0;
    const ClusterVariant* tab = pl->dt == RK_F32 ? cluster_variants_f32(&count)
                              : pl->dt == RK_BF16 ? cluster_variants_bf16(&count)
                                                  : cluster_variants_fp8(&count);
    // 128 consumers per CTA up to 1024 slices per chunk; 256 (up to 13 slices each, the
    // register budget of 9 warps) for the chunks of very long rows
    const int nt = chunk <= 128 * 8 ? 128 : 256;
    const int need = (chunk + nt - 1) / nt;
    int want_w = a.opts.lookahead > 1 ? a.opts.lookahead : 6;
    const ClusterVariant* var = nullptr;
    uint32_t stride = 0;
    int S = 0;
    for (int w : {want_w, 6, 4, 2}) {
        const ClusterVariant* best = nullptr;
        for (int i = 0; i < count; ++i)
            if (tab[i].nt == nt && tab[i].w == w && tab[i].vpt >= need && (!best || tab[i].vpt < best->vpt))
                best = &tab[i];
        if (!best) continue;
        const uint32_t bytes = (uint32_t)chunk * 4u * eb;
        const uint32_t padded = (uint32_t)nt * (uint32_t)best->vpt * 4u * eb;
        stride = ((bytes > padded ? bytes : padded) + 127u) & ~127u;
        S = 0;
        while (S < kMaxStages && (size_t)(S + 1) * stride + cluster_ctrl_bytes(S + 1, nt) <= (size_t)smem_max) ++S;
        if (S >= 2 * w) {
            var = best;
            break;
        }
    }
    if (!var) return RK_EINVAL;
    if (cudaFuncSetAttribute(var->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)S * stride + cluster_ctrl_bytes(S, nt))) != cudaSuccess)
        return RK_ECUDA;
    if (C > 8 && cudaFuncSetAttribute(var->fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return RK_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.q * C));
    cfg.blockDim = dim3((unsigned)(nt + 32));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // The grid barrier needs every CTA resident at once.  A deep ring can leave
    // one CTA per SM, and a GPC then holds fewer whole clusters: shorten the
    // ring (down to two groups) until the q clusters fit, else refuse.
    int clusters = 0;
    for (;;) {
        cfg.dynamicSmemBytes = (size_t)S * stride + cluster_ctrl_bytes(S, nt);
        if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)var->fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return RK_ECUDA;
        }
        if (clusters >= a.q || S <= 2 * var->w) break;
        --S;
    }
    if (clusters < a.q) return RK_ENOTCORESIDENT;
    CParams cp;
    cp.k = base;
    cp.k.stages = S;
    cp.k.stage_stride = stride;
    cp.k.row_bytes = 0;   // per-CTA copy sizes are computed in the kernel
    cp.chunk = chunk;
    if (cudaLaunchKernelEx(&cfg, var->fn, cp) != cudaSuccess) return RK_ECUDA;
    count_launch();
    return RK_OK;
}

static KParams base_params(const SolveArgs& a) {
    const Plan* pl = a.plan;
    KParams p{};
    p.A = static_cast<const uint8_t*>(pl->A);
    p.lda_bytes = pl->lda * (int64_t)elem_size(pl->dt);
    p.m = (uint64_t)pl->m;
    p.n = (int)pl->n;
    p.n4 = (int)((pl->n + 3) / 4);
    p.b = a.b;
    p.inv = pl->ws.inv;
    p.row_scale = pl->row_scale;
    p.thr64 = pl->ws.thr64;
    p.alias = pl->ws.alias;
    p.x0 = a.x0;
    p.x = a.x;
    p.V = a.V;
    p.ldv = a.ldv;
    const int rows = v_rows_for(a.q, a.alpha);
    p.xbuf = a.V + (size_t)rows * (size_t)a.ldv;
    p.chkpart = a.V + (size_t)(rows + 1) * (size_t)a.ldv;
    p.vrows = a.q;
    p.jacobi = 0;
    p.sampling = a.opts.sampling;
    p.P = pl->ws.P;
    p.row_weight = a.opts.row_weight;
    p.worker_weight = a.opts.worker_weight;
    p.q = a.q;
    p.alpha = a.alpha;
    p.rounds = a.rounds;
    p.round0 = a.opts.round0;
    p.seed = a.seed;
    p.stream_id = a.opts.stream_id;
    p.same_stream = a.opts.same_stream;
    p.omega = a.opts.omega;
    p.x_ref = a.opts.x_ref;
    p.tol = a.opts.tol;
    p.check_every = a.opts.check_every;
    p.criterion = a.opts.criterion;
    p.info = a.info;
    p.setup = pl->ws.info;
    p.timeout_ns = (uint64_t)(a.opts.timeout_s * 1e9);
    return p;
}

int launch_solve(const SolveArgs& a, cudaStream_t st) {
    const Plan* pl = a.plan;
    const int n4 = (int)((pl->n + 3) / 4);
    int dev = 0;
    cudaGetDevice(&dev);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (a.opts.cluster_size > 1) return launch_cluster_solve(a, base_params(a), a.opts.cluster_size, st, smem_max);
    // slices of 4 elements; the copy is rounded up to 16 bytes, which stays inside
    // the row's lda extent because lda * element size is a multiple of 16
    const uint32_t row_bytes = ((uint32_t)n4 * 4u * (uint32_t)elem_size(pl->dt) + 15u) & ~15u;
    // More workers than SMs: the two-per-SM variants (W = 1), each CTA within half
    // of the SM's shared memory (less the per-block reservation).
    int sms = 0, smem_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // RKA (alpha = 1) with more workers than SMs: the q single-projection workers
    // of a round are spread over one CTA per SM, each summing its workers'
    // projections from the round's x (their order inside the CTA does not matter:
    // they are independent, Eq. (rka_eq))
    const bool jac = a.alpha == 1 && a.q > sms;
    const int grid = jac ? sms : a.q;
    if (a.q > sms && !jac) {
        const SolveVariant* v2 = pick_variant(pl->dt, n4, 1, 2);
        if (!v2 || a.q > 2 * sms) return RK_ENOTCORESIDENT;
        const int half = smem_sm / 2 - 1024;
        const uint32_t padded2 = (uint32_t)v2->nt * (uint32_t)v2->vpt * 4u * (uint32_t)elem_size(pl->dt);
        const uint32_t stride2 = ((row_bytes > padded2 ? row_bytes : padded2) + 127u) & ~127u;
        const int S2 = stages_for(stride2, v2->nt, half < smem_max ? half : smem_max);
        if (S2 < 2) return RK_ENOTCORESIDENT;
        const size_t smem2 = (size_t)S2 * stride2 + solve_ctrl_bytes(S2, v2->nt);
        KParams p2 = base_params(a);
        p2.stages = S2;
        p2.row_bytes = row_bytes;
        p2.stage_stride = stride2;
        if (cudaFuncSetAttribute(v2->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) !=
            cudaSuccess)
            return RK_ECUDA;
        void* args2[] = {(void*)&p2};
        cudaError_t e2 = cudaLaunchCooperativeKernel((const void*)v2->fn, dim3((unsigned)a.q),
                                                     dim3((unsigned)(v2->nt + 32)), args2, smem2, st);
        if (e2 == cudaErrorCooperativeLaunchTooLarge) {
            cudaGetLastError();
            return RK_ENOTCORESIDENT;
        }
        if (e2 != cudaSuccess) return RK_ECUDA;
        count_launch();
        return RK_OK;
    }
    // look-ahead groups pay off when the per-row reduction outweighs the slice
    // work (short rows); the ring must hold two groups so that the producer fills
    // one while the consumers work on the other
    int w = jac ? 1 : a.opts.lookahead;
    const SolveVariant* var = nullptr;
    uint32_t stride = 0;
    int S = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
        const SolveVariant* v1 = pick_variant(pl->dt, n4, 1, 1, jac);
        if (!v1) break;   // no one-CTA variant holds the row
        // measured: groups of 4 pay off only with a single consumer warp (n <= 512);
        // from 128 consumers up, one row at a time is faster (0.34 against 0.40 us a
        // row at n = 1000, 0.43 against 0.63-0.66 at n = 4000)
        const int wauto = jac ? 1 : ((w == 0) ? (v1->nt == 32 ? 4 : 1) : w);
        var = pick_variant(pl->dt, n4, wauto, 1, jac);
        if (!var) var = v1;
        // stages are padded to the variant's NT * VPT slices (zeroed at kernel start)
        const uint32_t padded = (uint32_t)var->nt * (uint32_t)var->vpt * 4u * (uint32_t)elem_size(pl->dt);
        stride = ((row_bytes > padded ? row_bytes : padded) + 127u) & ~127u;
        S = stages_for(stride, var->nt, smem_max - (int)xs_bytes(var));
        if (S >= 2 * var->w) break;
        w = var->w > 1 ? var->w / 2 : 1;   // fewer rows per group when the ring is short
        var = nullptr;
    }
    if (!var || S < 2) {
        // a row too long for two stages of one CTA: RKA runs with x split by columns
        // over the grid (rk_colsplit.cu), every CTA streaming its chunk of each row
        if (colsplit_fits(a.alpha, a.q)) return launch_colsplit_solve(a, base_params(a), st, smem_max, sms);
        return RK_EINVAL;
    }
    const size_t smem = (size_t)S * stride + xs_bytes(var) + solve_ctrl_bytes(S, var->nt);

    KParams p = base_params(a);
    p.stages = S;
    p.row_bytes = row_bytes;
    p.stage_stride = stride;
    if (jac) {
        p.jacobi = 1;
        p.vrows = grid;
    }

    if (cudaFuncSetAttribute(var->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return RK_ECUDA;
    void* args[] = {(void*)&p};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)var->fn, dim3((unsigned)grid),
                                                dim3((unsigned)(var->nt + 32)), args, smem, st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        return RK_ENOTCORESIDENT;
    }
    if (e != cudaSuccess) return RK_ECUDA;
    count_launch();
    return RK_OK;
}

// Draws of one worker under any row selection (the draw_row of the solve kernels).
__global__ void sample_indices_ex_kernel(const KParams p, uint32_t worker, uint64_t t0, int64_t count,
                                         uint32_t* out) {
    if (p.setup->status != 0) return;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = draw_row(p, worker, t0 + (uint64_t)k);
}

int launch_sample_indices_ex(const Plan* plan, uint64_t seed, uint32_t worker, uint32_t q,
                             uint32_t stream_id, int sampling, uint64_t t0, int64_t count,
                             uint32_t* out, cudaStream_t st) {
    if (count <= 0) return RK_OK;
    KParams p{};
    p.m = (uint64_t)plan->m;
    p.seed = seed;
    p.stream_id = stream_id;
    p.thr64 = plan->ws.thr64;
    p.alias = plan->ws.alias;
    p.q = (int)q;
    p.sampling = sampling;
    p.P = plan->ws.P;
    p.setup = plan->ws.info;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    sample_indices_ex_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, worker, t0, count, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

int launch_sample_indices(const Plan* plan, uint64_t seed, uint32_t worker, uint32_t stream_id,
                          uint64_t t0, int64_t count, uint32_t* out, cudaStream_t st) {
    if (count <= 0) return RK_OK;
    const int threads = 256;
    int64_t blocks = (count + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    sample_indices_kernel<<<(unsigned)blocks, threads, 0, st>>>(
        plan->ws.thr64, plan->ws.alias, (uint64_t)plan->m, seed, worker, stream_id, t0, count, out,
        plan->ws.info);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

static int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 256;
}

// Rows of V a solve with q workers may need whatever alpha is: one per CTA that holds
// displacements -- q for one or two workers per SM and for cluster workers (q is then
// at most twice the SM count), the SM count when RKA spreads more workers over the CTAs.
int v_rows(int q) {
    const int sms = device_sms();
    return q < 2 * sms ? q : 2 * sms;
}

// Rows of V the launch for (q, alpha) uses: the SM count for RKA with more workers than
// SMs (one CTA per SM sums its share of the workers), else q.
int v_rows_for(int q, int64_t alpha) {
    const int sms = device_sms();
    if (alpha == 1 && q > sms) return sms;
    return q < 2 * sms ? q : 2 * sms;
}

static size_t ws_bytes_rows(const Plan* plan, int rows) {
    const int64_t n4 = (plan->n + 3) / 4;
    const int64_t ldv = n4 * 4;
    // status | V (rows x ldv) and the average (ldv) | per-CTA check partials (a float4
    // for each of up to kClusterMax CTAs per row of V)
    return align256(sizeof(SolveInfo)) + align256((size_t)(rows + 1) * (size_t)ldv * sizeof(float) +
                                                  (size_t)rows * kClusterMax * 4 * sizeof(float));
}

size_t solve_ws_bytes(const Plan* plan, int q) { return ws_bytes_rows(plan, v_rows(q)); }

size_t solve_ws_bytes_for(const Plan* plan, int q, int64_t alpha) {
    return ws_bytes_rows(plan, v_rows_for(q, alpha));
}

}  // namespace rk
