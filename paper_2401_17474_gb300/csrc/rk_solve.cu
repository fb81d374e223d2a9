// rk_solve.cu -- persistent RKAB kernel (Section 3.4.1, Algorithm 3; alpha = 1
// is RKA, Algorithm 1 / Eq. (rka_uni_weights); q = 1 is RK, Eq. (alg) with the
// draws of Eq. (prob_line)).
//
// One CTA per worker gamma.  Warp layout of a CTA:
//   warps 0 .. NT/32-1  consumers: each thread owns VPT float4 slices of the
//                       round's start point x and of the worker's displacement
//                       d = v - x (registers) and, per projection, the
//                       matching slices of the sampled row;
//   warp NT/32          producer: draws the row indices ahead (they do not
//                       depend on v), loads b_i and 1/||A_i||^2 and moves each
//                       row HBM -> shared memory with one bulk asynchronous
//                       copy into a ring of `stages` buffers (mbarrier
//                       full/empty handshake).
// Per projection the consumers compute <A_i, v> = <A_i, x> + <A_i, d>
// (per-thread FMA chain, warp butterfly, fixed-order sum of the warp
// partials), the scale omega (b_i - <A_i, v>) / ||A_i||^2, and d += scale A_i,
// with one named barrier.  After `alpha` projections every CTA writes d to row
// gamma of V, a grid barrier follows, each CTA forms x + (1/q) sum_gamma d_gamma
// for a slice of columns, a second grid barrier follows, and every CTA reloads
// x and clears d.  Every wait is bounded in time.
//
// The worker keeps v as x + d, the difference form of Algorithm 3 (v - x is
// what gets averaged): near convergence a projection changes v_j by far less
// than half an ulp of v_j, so an iterate stored whole in float32 stops moving
// (stagnation near 1e-6 relative error on the 80000 x 10000 system); d is small
// and keeps the updates, and x is rounded once per round.
#include <algorithm>
#include <cstdint>

#include "rk_common.cuh"
#include "rk_internal.h"

namespace rk {

struct KParams {
    const float* A;
    int64_t lda;
    uint64_t m;
    int n;
    int n4;
    const float* b;
    const float* inv;
    const uint64_t* thr64;
    const uint32_t* alias;
    const float* x0;
    float* x;
    float* xbuf;        // n4 float4, the average (workspace)
    float* V;           // q x ldv
    int64_t ldv;
    int q;
    int64_t alpha;
    int64_t rounds;
    int64_t round0;
    uint64_t seed;
    uint32_t stream_id;
    int same_stream;
    float omega;
    const float* x_ref;
    double tol;
    int64_t check_every;
    int criterion;
    SolveInfo* info;
    const SetupInfo* setup;
    uint64_t timeout_ns;
    int stages;
    uint32_t row_bytes;     // bytes moved per row (n4 * 16)
    uint32_t stage_stride;  // bytes between stages in shared memory
};

struct Ctrl {
    long long stop_t;   // producer issues projections t < stop_t
    int flag;           // broadcast slot
    int pad;
};

__device__ __forceinline__ bool bar_and(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity, uint64_t timeout_ns,
                                            int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > timeout_ns) {
            set_status(status, RK_ETIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ float4 ldcg4(const float* p) {
    return __ldcg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ float4 mask_tail(float4 v, int idx, int n4, int n) {
    const int rem = n & 3;
    if (rem && idx == n4 - 1) {
        if (rem < 2) v.y = 0.f;
        if (rem < 3) v.z = 0.f;
        v.w = 0.f;
    }
    return v;
}

template <int NT>
__device__ void producer_loop(const KParams& p, uint8_t* stages, uint64_t* full, uint64_t* empty,
                              float2* meta, volatile Ctrl* ctrl) {
    const int lane = threadIdx.x & 31;
    const int S = p.stages;
    const int64_t total = p.rounds * p.alpha;
    const uint32_t worker = p.same_stream ? 0u : (uint32_t)blockIdx.x;
    const uint64_t tbase = (uint64_t)p.round0 * (uint64_t)p.alpha;
    const uint64_t pol = policy_evict_first();
    int* status = &p.info->status;
    int64_t issued = 0;
    int s = 0;
    uint32_t pass = 0;      // parity of the current pass over the ring of stages
    bool stop = false;
    for (int64_t base = 0; base < total && !stop; base += 32) {
        const int64_t tl = base + lane;
        uint32_t row = 0;
        float bi = 0.f, iv = 0.f;
        if (tl < total) {
            row = sample_row(p.seed, worker, p.stream_id, tbase + (uint64_t)tl, p.m, p.thr64, p.alias);
            bi = __ldg(p.b + row);
            iv = __ldg(p.inv + row);
        }
        const int64_t rem_ = total - base;
        const int cnt = rem_ < 32 ? (int)rem_ : 32;
        for (int k = 0; k < cnt; ++k) {
            const uint32_t rk_ = __shfl_sync(0xffffffffu, row, k);
            const float bk = __shfl_sync(0xffffffffu, bi, k);
            const float ik = __shfl_sync(0xffffffffu, iv, k);
            if (lane == 0) {
                const int64_t tt = base + k;
                if (tt >= ctrl->stop_t) {
                    stop = true;
                } else {
                    if (tt >= S) {
                        // wait until the consumers released this stage's row of the
                        // previous pass (phase parity = previous pass parity)
                        const uint32_t prev = pass ^ 1u;
                        if (!mbar_try_wait(&empty[s], prev)) {
                            const uint64_t t0 = globaltimer_ns();
                            while (!mbar_try_wait(&empty[s], prev)) {
                                if (tt >= ctrl->stop_t) { stop = true; break; }
                                if (globaltimer_ns() - t0 > p.timeout_ns) {
                                    set_status(status, RK_ETIMEOUT);
                                    stop = true;
                                    break;
                                }
                            }
                        }
                    }
                    if (!stop) {
                        meta[s] = make_float2(bk, ik);
                        mbar_arrive_expect_tx(&full[s], p.row_bytes);
                        bulk_g2s(stages + (size_t)s * p.stage_stride,
                                 p.A + (size_t)rk_ * (size_t)p.lda, p.row_bytes, &full[s], pol);
                        issued = tt + 1;
                        if (++s == S) { s = 0; pass ^= 1u; }
                    }
                }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) break;
        }
    }
    // Drain: every copy this warp issued must have landed before the CTA exits.
    if (lane == 0) {
        const int64_t first = issued > S ? issued - S : 0;
        for (int64_t tt = first; tt < issued; ++tt) {
            const int st = (int)(tt % S);
            const uint32_t par = (uint32_t)((tt / S) & 1);
            wait_parity(&full[st], par, p.timeout_ns, status);
        }
    }
    __syncwarp();
}

// x <- x + (1/q) sum_gamma d_gamma (d_gamma = V[gamma]) for this CTA's
// contiguous slice of float4 columns; x is read from x0 in the first round and
// from xbuf afterwards (only the slice's owner reads and writes it here).  When the slice is narrower than the CTA, the workers are split into
// `groups` contiguous ranges, each summed in ascending gamma by one thread, and
// the group sums are added in ascending group order: a fixed two-level order,
// the same on every run.  Writes the average to xbuf (float4) and to x.
__device__ __forceinline__ float4 load_x_old(const KParams& p, int c, bool first) {
    if (!first) return ldcg4(p.xbuf + (size_t)c * 4);
    const int j = c * 4;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    t.x = p.x0[j];
    if (j + 1 < p.n) t.y = p.x0[j + 1];
    if (j + 2 < p.n) t.z = p.x0[j + 2];
    if (j + 3 < p.n) t.w = p.x0[j + 3];
    return t;
}

__device__ __forceinline__ void store_x(const KParams& p, int c, float4 xm) {
    reinterpret_cast<float4*>(p.xbuf)[c] = xm;
    const int j = c * 4;
    p.x[j] = xm.x;
    if (j + 1 < p.n) p.x[j + 1] = xm.y;
    if (j + 2 < p.n) p.x[j + 2] = xm.z;
    if (j + 3 < p.n) p.x[j + 3] = xm.w;
}

template <int NT>
__device__ __forceinline__ void average_slice(const KParams& p, float4* avg, bool first) {
    const int tid = threadIdx.x;
    const int n4 = p.n4;
    const int G = gridDim.x;
    const int cols = (n4 + G - 1) / G;
    const int c0 = blockIdx.x * cols;
    const int c1 = min(n4, c0 + cols);
    const int nc = c1 - c0;
    const float qf = (float)p.q;
    if (nc <= 0) return;
    if (nc >= NT) {
        for (int c = c0 + tid; c < c1; c += NT) {
            float4 acc = ldcg4(p.V + (size_t)c * 4);
#pragma unroll 8
            for (int g = 1; g < p.q; ++g) {
                const float4 w = ldcg4(p.V + (size_t)g * (size_t)p.ldv + (size_t)c * 4);
                acc.x += w.x; acc.y += w.y; acc.z += w.z; acc.w += w.w;
            }
            const float4 xo = load_x_old(p, c, first);
            store_x(p, c, make_float4(xo.x + acc.x / qf, xo.y + acc.y / qf, xo.z + acc.z / qf,
                                      xo.w + acc.w / qf));
        }
        return;
    }
    int groups = NT / nc;
    if (groups > p.q) groups = p.q;
    const int per = (p.q + groups - 1) / groups;
    const int cl = tid % nc, g = tid / nc;
    if (g < groups) {
        const int ga = g * per, gb = min(p.q, ga + per);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int gg = ga; gg < gb; ++gg) {
            const float4 w = ldcg4(p.V + (size_t)gg * (size_t)p.ldv + (size_t)(c0 + cl) * 4);
            acc.x += w.x; acc.y += w.y; acc.z += w.z; acc.w += w.w;
        }
        avg[g * nc + cl] = acc;
    }
    named_bar_sync(1, NT);
    if (tid < nc) {
        float4 acc = avg[tid];
        for (int gg = 1; gg < groups; ++gg) {
            const float4 w = avg[gg * nc + tid];
            acc.x += w.x; acc.y += w.y; acc.z += w.z; acc.w += w.w;
        }
        const int c = c0 + tid;
        const float4 xo = load_x_old(p, c, first);
        store_x(p, c, make_float4(xo.x + acc.x / qf, xo.y + acc.y / qf, xo.z + acc.z / qf,
                                  xo.w + acc.w / qf));
    }
}

template <int NT, int VPT>
__global__ void __launch_bounds__(NT + 32, 1) rkab_kernel(const KParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int NW = NT / 32;
    const int S = p.stages;
    uint8_t* stages = smem;
    // tail of shared memory: see ctrl_bytes()
    float4* avg = reinterpret_cast<float4*>(smem + (size_t)S * p.stage_stride);  // [NT]
    uint64_t* full = reinterpret_cast<uint64_t*>(avg + NT);
    uint64_t* empty = full + S;
    float2* meta = reinterpret_cast<float2*>(empty + S);
    float* red = reinterpret_cast<float*>(meta + S);          // [2][32] dot partials
    double* chk = reinterpret_cast<double*>(red + 64);        // [3][32] check partials
    volatile Ctrl* ctrl = reinterpret_cast<volatile Ctrl*>(chk + 96);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t total = p.rounds * p.alpha;
    int* status = &p.info->status;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        ctrl->stop_t = total;
        ctrl->flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (p.setup->status != 0) {
        if (tid == 0) set_status(status, RK_ESETUP);
        return;
    }
    if (warp == NW) {
        producer_loop<NT>(p, stages, full, empty, meta, ctrl);
        return;
    }

    // ---------------- consumers ----------------
    const int n4 = p.n4;
    const int gamma = blockIdx.x;
    float4 v[VPT];   // the round's start point x
    float4 d[VPT];   // the worker's displacement v - x within the round
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        const int idx = tid + k * NT;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < n4) {
            const int j = idx * 4;
            t.x = __ldg(p.x0 + j);
            if (j + 1 < p.n) t.y = __ldg(p.x0 + j + 1);
            if (j + 2 < p.n) t.z = __ldg(p.x0 + j + 2);
            if (j + 3 < p.n) t.w = __ldg(p.x0 + j + 3);
        }
        v[k] = t;
        d[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    int s = 0;
    uint32_t ph = 0;
    int rp = 0;
    int64_t t = 0;
    bool ok = true;
    float* Vg = p.V + (size_t)gamma * (size_t)p.ldv;
    for (int64_t r = 0; r < p.rounds && ok; ++r) {
        for (int64_t j = 0; j < p.alpha; ++j, ++t) {
            const bool got = wait_parity(&full[s], ph, p.timeout_ns, status);
            const float4* st4 = reinterpret_cast<const float4*>(stages + (size_t)s * p.stage_stride);
            float4 a[VPT];
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int idx = tid + k * NT;
                a[k] = (idx < n4) ? mask_tail(st4[idx], idx, n4, p.n) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const float2 mb = meta[s];
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            float part = 0.f;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                part = fmaf(a[k].x, v[k].x, part);
                part = fmaf(a[k].x, d[k].x, part);
                part = fmaf(a[k].y, v[k].y, part);
                part = fmaf(a[k].y, d[k].y, part);
                part = fmaf(a[k].z, v[k].z, part);
                part = fmaf(a[k].z, d[k].z, part);
                part = fmaf(a[k].w, v[k].w, part);
                part = fmaf(a[k].w, d[k].w, part);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) red[rp * 32 + warp] = part;
            if (!bar_and(1, NT, got)) { ok = false; break; }
            float dot = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) dot += red[rp * 32 + w];
            rp ^= 1;
            const float scale = p.omega * (mb.x - dot) * mb.y;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                d[k].x = fmaf(scale, a[k].x, d[k].x);
                d[k].y = fmaf(scale, a[k].y, d[k].y);
                d[k].z = fmaf(scale, a[k].z, d[k].z);
                d[k].w = fmaf(scale, a[k].w, d[k].w);
            }
            if (++s == p.stages) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;

        // ---- average: x <- x + (1/q) sum_gamma d_gamma ----
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int idx = tid + k * NT;
            if (idx < n4) reinterpret_cast<float4*>(Vg)[idx] = d[k];
        }
        named_bar_sync(1, NT);
        if (tid == 0) ctrl->flag = grid_barrier(&p.info->bar_count, &p.info->bar_gen, gridDim.x,
                                                 status, p.timeout_ns) ? 1 : 0;
        named_bar_sync(1, NT);
        if (!ctrl->flag) { ok = false; break; }
        average_slice<NT>(p, avg, r == 0);
        named_bar_sync(1, NT);
        if (tid == 0) ctrl->flag = grid_barrier(&p.info->bar_count, &p.info->bar_gen, gridDim.x,
                                                 status, p.timeout_ns) ? 1 : 0;
        named_bar_sync(1, NT);
        if (!ctrl->flag) { ok = false; break; }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int idx = tid + k * NT;
            v[k] = (idx < n4) ? ldcg4(p.xbuf + (size_t)idx * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
            d[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }

        // ---- convergence / divergence check (identical in every CTA) ----
        const int64_t done = r + 1;
        const bool last = (done == p.rounds);
        if (p.check_every > 0 && (done % p.check_every == 0 || last)) {
            float e2 = 0.f, r2 = 0.f, xx = 0.f;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int idx = tid + k * NT;
                if (idx < n4) {
                    xx = fmaf(v[k].x, v[k].x, xx);
                    xx = fmaf(v[k].y, v[k].y, xx);
                    xx = fmaf(v[k].z, v[k].z, xx);
                    xx = fmaf(v[k].w, v[k].w, xx);
                    if (p.criterion == 1) {
                        const int j0 = idx * 4;
                        const float vv[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (j0 + c < p.n) {
                                const float xr = __ldg(p.x_ref + j0 + c);
                                const float d = vv[c] - xr;
                                e2 = fmaf(d, d, e2);
                                r2 = fmaf(xr, xr, r2);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                e2 += __shfl_xor_sync(0xffffffffu, e2, o);
                r2 += __shfl_xor_sync(0xffffffffu, r2, o);
                xx += __shfl_xor_sync(0xffffffffu, xx, o);
            }
            if (lane == 0) {
                chk[warp] = (double)e2;
                chk[32 + warp] = (double)r2;
                chk[64 + warp] = (double)xx;
            }
            named_bar_sync(1, NT);
            double E2 = 0.0, R2 = 0.0, XX = 0.0;
            for (int w = 0; w < NW; ++w) {
                E2 += chk[w];
                R2 += chk[32 + w];
                XX += chk[64 + w];
            }
            named_bar_sync(1, NT);
            double metric = -1.0;
            if (p.criterion == 1) metric = (R2 > 0.0) ? sqrt(E2 / R2) : sqrt(E2);
            const bool diverged = !isfinite(XX) || (p.criterion == 1 && !isfinite(metric));
            if (gamma == 0 && tid == 0) {
                p.info->rounds_done = done;
                p.info->last_metric = metric;
            }
            if (diverged) {
                if (tid == 0) set_status(status, RK_EDIVERGED);
                ok = false;
            } else if (p.criterion == 1 && p.tol > 0.0 && metric < p.tol) {
                break;  // converged: identical decision in every CTA
            }
        } else if (gamma == 0 && tid == 0) {
            p.info->rounds_done = done;
        }
    }
    // Stop the producer at what was consumed (no-op after the last round).
    if (tid == 0) ctrl->stop_t = t;
}

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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef void (*KernelFn)(const KParams);

struct Variant {
    int nt, vpt;
    KernelFn fn;
};

#define RK_VARIANT(NT, VPT) Variant{NT, VPT, rkab_kernel<NT, VPT>}
static const Variant kVariants[] = {
    RK_VARIANT(32, 1),  RK_VARIANT(32, 2),  RK_VARIANT(32, 4),
    RK_VARIANT(128, 2), RK_VARIANT(128, 3), RK_VARIANT(128, 4), RK_VARIANT(128, 5),
    RK_VARIANT(512, 2), RK_VARIANT(512, 3), RK_VARIANT(512, 4), RK_VARIANT(512, 5),
    RK_VARIANT(512, 6), RK_VARIANT(512, 8), RK_VARIANT(512, 10),
};
#undef RK_VARIANT

static const Variant* pick_variant(int n4) {
    int nt = n4 <= 32 * 4 ? 32 : (n4 <= 128 * 5 ? 128 : 512);
    const int need = (n4 + nt - 1) / nt;
    for (const Variant& v : kVariants) {
        if (v.nt == nt && v.vpt >= need) return &v;
    }
    return nullptr;
}

static const int kMaxStages = 16;

// avg[NT] float4, full[S] + empty[S] mbarriers, meta[S] float2, red[64] float,
// chk[96] double, Ctrl.
static size_t ctrl_bytes(int S, int nt) {
    return (size_t)nt * 16 + (size_t)S * 24 + 64 * 4 + 96 * 8 + 64;
}

int launch_solve(const SolveArgs& a, cudaStream_t st) {
    const Plan* pl = a.plan;
    if (pl->dt != RK_F32) return RK_EINVAL;  // stored-precision solves use their own kernels
    const int n4 = (int)((pl->n + 3) / 4);
    const Variant* var = pick_variant(n4);
    if (!var) return RK_EINVAL;
    int dev = 0;
    cudaGetDevice(&dev);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const uint32_t row_bytes = (uint32_t)n4 * 16u;
    const uint32_t stride = (row_bytes + 127u) & ~127u;
    int S = 0;
    while (S < kMaxStages && (size_t)(S + 1) * stride + ctrl_bytes(S + 1, var->nt) <= (size_t)smem_max) ++S;
    if (S < 2) return RK_EINVAL;
    const size_t smem = (size_t)S * stride + ctrl_bytes(S, var->nt);

    KParams p{};
    p.A = static_cast<const float*>(pl->A);
    p.lda = pl->lda;
    p.m = (uint64_t)pl->m;
    p.n = (int)pl->n;
    p.n4 = n4;
    p.b = a.b;
    p.inv = pl->ws.inv;
    p.thr64 = pl->ws.thr64;
    p.alias = pl->ws.alias;
    p.x0 = a.x0;
    p.x = a.x;
    p.V = a.V;
    p.ldv = a.ldv;
    p.xbuf = a.V + (size_t)a.q * (size_t)a.ldv;
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
    p.stages = S;
    p.row_bytes = row_bytes;
    p.stage_stride = stride;

    if (cudaFuncSetAttribute(var->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return RK_ECUDA;
    void* args[] = {(void*)&p};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)var->fn, dim3((unsigned)a.q),
                                                dim3((unsigned)(var->nt + 32)), args, smem, st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        return RK_ENOTCORESIDENT;
    }
    if (e != cudaSuccess) return RK_ECUDA;
    count_launch();
    return RK_OK;
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

size_t solve_ws_bytes(const Plan* plan, int q) {
    const int64_t n4 = (plan->n + 3) / 4;
    const int64_t ldv = n4 * 4;
    return align256(sizeof(SolveInfo)) + align256((size_t)(q + 1) * (size_t)ldv * sizeof(float));
}

}  // namespace rk
