// rk_solve_kernel.cuh -- persistent RKAB kernel (Section 3.4.1, Algorithm 3;
// alpha = 1 is RKA, Algorithm 1 / Eq. (rka_uni_weights); q = 1 is RK,
// Eq. (alg) with the draws of Eq. (prob_line)), templated on the stored row
// type (float32, bfloat16, FP8 e4m3 with a per-row scale).  Instantiated in
// rk_solve_f32.cu, rk_solve_bf16.cu and rk_solve_fp8.cu; launched by rk_solve.cu.
//
// One CTA per worker gamma.  Warp layout of a CTA:
//   warps 0 .. NT/32-1  consumers: each thread owns VPT four-element slices of
//                       the round's start point x and of the worker's
//                       displacement d = v - x (registers, float32) and, per
//                       projection, the matching elements of the sampled row;
//   warp NT/32          producer: draws the row indices ahead (they do not
//                       depend on v), loads b_i, 1/||A_i||^2 (and the FP8 row
//                       scale) and moves each stored row HBM -> shared memory
//                       with one bulk asynchronous copy into a ring of
//                       `stages` buffers (mbarrier full/empty handshake).
// Per projection the consumers compute <A_i, v> = <A_i, x> + <A_i, d>
// (per-thread FMA chain, warp butterfly, fixed-order sum of the warp
// partials), the scale omega (b_i - <A_i, v>) / ||A_i||^2, and d += scale A_i,
// with one named barrier.  Rows stored in BF16 or FP8 are widened to float32
// in registers; the FP8 row scale s_i multiplies the dot and the update scalar
// (A_i = s_i q_i), so the arithmetic stays float32.  After `alpha`
// projections every CTA writes d to row gamma of V, a grid barrier follows,
// each CTA forms x + (1/q) sum_gamma d_gamma for a slice of columns, a second
// grid barrier follows, and every CTA reloads x and clears d.  Every wait is
// bounded in time.
//
// The worker keeps v as x + d, the difference form of Algorithm 3 (v - x is
// what gets averaged): near convergence a projection changes v_j by far less
// than half an ulp of v_j, so an iterate stored whole in float32 stops moving
// (stagnation near 1e-6 relative error on the 80000 x 10000 system); d is small
// and keeps the updates, and x is rounded once per round.
//
// KEEP_A: the row's slices stay in registers between the dot and the update
// (the stage is released right after it is read).  Without it (wide rows, where
// x, d and the row together would not fit in registers) the update reads the
// stage a second time and the stage is released after the update.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>

#include "rk_common.cuh"
#include "rk_internal.h"

namespace rk {

enum { ELT_F32 = 0, ELT_BF16 = 1, ELT_FP8 = 2 };

struct KParams {
    const uint8_t* A;       // stored rows
    int64_t lda_bytes;
    uint64_t m;
    int n;
    int n4;                 // ceil(n / 4): four-element slices per row
    const float* b;
    const float* inv;
    const float* row_scale; // FP8 only
    const uint64_t* thr64;
    const uint32_t* alias;
    const float* x0;
    float* x;
    float* xbuf;            // n4 float4, the average (workspace)
    float* V;               // q x ldv
    int64_t ldv;
    float* chkpart;         // gridDim.x float4: per-CTA check partials of its x slice
    int vrows;              // rows of V holding displacements (averaged, divided by q)
    int sampling;           // rk_sampling: full law, per-worker row blocks, cyclic
    const uint64_t* P;      // exclusive prefix of the integer weights (row blocks)
    const float* row_weight;  // per-row weights w_i (NULL: 1)
    const float* worker_weight;  // per-worker weights (NULL: 1)
    int jacobi;             // RKA with q workers spread over the CTAs (alpha = 1): CTA g
                            // holds workers [g q / G, (g+1) q / G), each one projection per
                            // round from the round's x; their sum is the CTA's row of V
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
    uint32_t row_bytes;     // bytes moved per row (multiple of 16)
    uint32_t stage_stride;  // bytes between stages in shared memory
};

// Row of worker `worker` (of q) at projection counter t under the sampling mode:
// the alias draw of the full law; the Distributed Approach's block draw (Philox
// words as for the alias draw; c = floor(u T_g / 2^64) picks the row whose prefix
// interval [P_i, P_i + K_i) holds P_start + c, found by bisection; returns m for a
// block of zero weight); or the cyclic sweep from the block's first row.
__device__ __forceinline__ uint32_t draw_row(const KParams& p, uint32_t worker, uint64_t t) {
    if (p.sampling == RK_SAMPLE_FULL)
        return sample_row(p.seed, worker, p.stream_id, t, p.m, p.thr64, p.alias);
    const uint64_t q = (uint64_t)p.q, g = worker;
    const uint64_t start = (g * p.m) / q, end = ((g + 1) * p.m) / q;
    if (p.sampling == RK_SAMPLE_CYCLIC) return (uint32_t)((start + t) % p.m);
    const uint64_t ps = __ldg(p.P + start);
    const uint64_t pe = end == p.m ? p.setup->T : __ldg(p.P + end);
    const uint64_t tg = pe - ps;
    if (tg == 0 || end <= start) return (uint32_t)p.m;
    const U4 r = philox10(U4{(uint32_t)t, (uint32_t)(t >> 32), worker, p.stream_id},
                          (uint32_t)p.seed, (uint32_t)(p.seed >> 32));
    const uint64_t u = (uint64_t)r.x | ((uint64_t)r.y << 32);
    const uint64_t target = ps + __umul64hi(u, tg);
    uint64_t lo = start, hi = end - 1;   // the largest i in the block with P_i <= target
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(p.P + mid) <= target) lo = mid;
        else hi = mid - 1;
    }
    return (uint32_t)lo;
}

// Projections a CTA makes per round: alpha, or with JAC its share of the q workers
// (CTA g holds workers [g q / G, (g+1) q / G)).
template <bool JAC>
__device__ __forceinline__ int cta_projections(const KParams& p) {
    if constexpr (!JAC) {
        return (int)p.alpha;
    } else {
        const int G = (int)gridDim.x;
        return (int)(((blockIdx.x + 1) * p.q) / G - (blockIdx.x * p.q) / G);
    }
}

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

// Sum of the NW warp partials of one slot of `red` (NW a power of two, the slot 16-byte
// aligned), computed by every thread from vector loads of shared memory in the order of
// a butterfly over the partials read by lane 0 (pairs at distance NW/2, then NW/4, ...):
// the same value, bit for bit, in every thread, without shuffles.
template <int NW>
__device__ __forceinline__ float cta_sum(const float* slot) {
    static_assert((NW & (NW - 1)) == 0 && NW <= 32, "warp count");
    float t[NW];
    if constexpr (NW >= 4) {
#pragma unroll
        for (int i = 0; i < NW / 4; ++i) {
            const float4 v = reinterpret_cast<const float4*>(slot)[i];
            t[4 * i] = v.x; t[4 * i + 1] = v.y; t[4 * i + 2] = v.z; t[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NW; ++i) t[i] = slot[i];
    }
#pragma unroll
    for (int o = NW / 2; o >= 1; o >>= 1) {
#pragma unroll
        for (int l = 0; l < o; ++l) t[l] = t[l] + t[l + o];
    }
    return t[0];
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

// Zero the elements of the row's last slice that lie beyond column n (they are
// copied from the row's padding).  rem = n mod 4 (nonzero here).
__device__ __forceinline__ float4 zero_beyond(float4 v, int rem) {
    if (rem < 2) v.y = 0.f;
    if (rem < 3) v.z = 0.f;
    v.w = 0.f;
    return v;
}

template <int ELT>
__device__ __forceinline__ float4 load4(const uint8_t* stage, int idx) {
    if constexpr (ELT == ELT_F32) {
        return reinterpret_cast<const float4*>(stage)[idx];
    } else if constexpr (ELT == ELT_BF16) {
        const uint2 w = reinterpret_cast<const uint2*>(stage)[idx];
        return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xFFFF0000u),
                           __uint_as_float(w.y << 16), __uint_as_float(w.y & 0xFFFF0000u));
    } else {
        const uint32_t w = reinterpret_cast<const uint32_t*>(stage)[idx];
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
        const float2 a = __half22float2(__half2(lo));
        const float2 c = __half22float2(__half2(hi));
        return make_float4(a.x, a.y, c.x, c.y);
    }
}

// Slice k of this thread as stored in the stage.  Stages are padded to NT*VPT
// slices and zeroed once when the kernel starts (copies never write beyond the
// row), so slices past the row read zeros and need no bounds check; only the
// row's last slice, when n is not a multiple of 4, is masked (tail_k is the k
// of that slice for the one thread that owns it, -1 elsewhere).
template <int ELT>
__device__ __forceinline__ float4 slice(const uint8_t* stg, int idx, int k, int tail_k, int rem) {
    float4 a = load4<ELT>(stg, idx);
    if (k == tail_k) a = zero_beyond(a, rem);
    return a;
}

// Four stored elements of slice idx of a stage, widened to float32 (the FP8 row
// scale is not applied here).
template <int ELT, bool JAC>
__device__ void producer_loop(const KParams& p, uint8_t* stages, uint64_t* full, uint64_t* empty,
                              float4* meta, volatile Ctrl* ctrl, float4* pbuf) {
    const int lane = threadIdx.x & 31;
    const int S = p.stages;
    const int per = cta_projections<JAC>(p);
    const int64_t total = p.rounds * (int64_t)per;
    const uint32_t worker = p.same_stream ? 0u : (uint32_t)blockIdx.x;
    const uint64_t tbase = (uint64_t)p.round0 * (uint64_t)p.alpha;
    const uint32_t w0 = JAC ? (uint32_t)((blockIdx.x * p.q) / (int)gridDim.x) : 0u;
    const uint64_t pol = policy_evict_first();
    int* status = &p.info->status;
    int64_t issued = 0;
    int s = 0;
    uint32_t pass = 0;      // parity of the current pass over the ring of stages
    bool stop = false;
    for (int64_t base = 0; base < total && !stop; base += 32) {
        // the warp draws 32 rows at once (their indices do not depend on v) ...
        const int64_t tl = base + lane;
        if (tl < total) {
            // worker gamma's t-th draw; with jacobi, draw j of round r belongs to
            // worker w0 + j and is its round0 + r-th projection
            uint32_t wk = worker;
            uint32_t own = blockIdx.x;   // the worker whose projection this is
            uint64_t tt = tbase + (uint64_t)tl;
            if constexpr (JAC) {
                own = w0 + (uint32_t)(tl % per);
                wk = p.same_stream ? 0u : own;
                tt = (uint64_t)p.round0 + (uint64_t)(tl / per);
            }
            uint32_t row = draw_row(p, wk, tt);
            if (row >= p.m) {   // a row block of zero weight: nothing to draw
                set_status(&p.info->status, RK_EINVAL);
                row = 0;
            }
            const float sc = (ELT == ELT_FP8) ? __ldg(p.row_scale + row) : 1.f;
            // a per-row weight w_i and a per-worker weight scale the projection with 1/||A_i||^2
            float wi = p.row_weight ? __ldg(p.row_weight + row) : 1.f;
            if (p.worker_weight) wi *= __ldg(p.worker_weight + own);
            pbuf[lane] = make_float4(__uint_as_float(row), __ldg(p.b + row), __ldg(p.inv + row) * wi, sc);
        }
        __syncwarp();
        // ... and one lane moves them, in order, into the ring of stages
        if (lane == 0) {
            const int64_t rem_ = total - base;
            const int cnt = rem_ < 32 ? (int)rem_ : 32;
            for (int k = 0; k < cnt && !stop; ++k) {
                const int64_t tt = base + k;
                if (tt >= ctrl->stop_t) {
                    stop = true;
                    break;
                }
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
                    if (stop) break;
                }
                const float4 e = pbuf[k];
                const uint32_t row = __float_as_uint(e.x);
                meta[s] = make_float4(e.y, e.z, e.w, 0.f);
                mbar_arrive_expect_tx(&full[s], p.row_bytes);
                bulk_g2s(stages + (size_t)s * p.stage_stride, p.A + (size_t)row * (size_t)p.lda_bytes,
                         p.row_bytes, &full[s], pol);
                issued = tt + 1;
                if (++s == S) { s = 0; pass ^= 1u; }
            }
        }
        stop = __shfl_sync(0xffffffffu, stop, 0);
        __syncwarp();
    }
    // Drain: every copy this warp issued must have landed before the CTA exits.
    if (lane == 0) {
        const int64_t first = issued > S ? issued - S : 0;
        for (int64_t tt = first; tt < issued; ++tt) {
            const int st = (int)(tt % S);
            const uint32_t par = (uint32_t)((tt / S) & 1);
            wait_parity(&full[st], par, drain_limit_ns(p.timeout_ns), status);
        }
    }
    __syncwarp();
}

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

// Partial sums of the convergence check over the columns a thread stores:
// ||x||^2 (divergence), and for criterion 1 ||x - x_ref||^2 and ||x_ref||^2.
// Float32 sums over a few elements each, combined by fixed-order trees: the
// check decides a relative error of 1e-6 or more, far above their rounding.
struct ChkAcc {
    float xx, e2, r2;
};

// The reference solution's slice c (elements past n read as 0), loaded before the
// column sums so that its latency overlaps theirs.
__device__ __forceinline__ float4 load_xref(const KParams& p, int c, bool want) {
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (want && p.criterion == 1) {
        const int j = c * 4;
        t.x = __ldg(p.x_ref + j);
        if (j + 1 < p.n) t.y = __ldg(p.x_ref + j + 1);
        if (j + 2 < p.n) t.z = __ldg(p.x_ref + j + 2);
        if (j + 3 < p.n) t.w = __ldg(p.x_ref + j + 3);
    }
    return t;
}

__device__ __forceinline__ void store_x(const KParams& p, int c, float4 xm, ChkAcc* acc, float4 xr4) {
    reinterpret_cast<float4*>(p.xbuf)[c] = xm;
    const int j = c * 4;
    p.x[j] = xm.x;
    if (j + 1 < p.n) p.x[j + 1] = xm.y;
    if (j + 2 < p.n) p.x[j + 2] = xm.z;
    if (j + 3 < p.n) p.x[j + 3] = xm.w;
    if (acc) {
        const float vv[4] = {xm.x, xm.y, xm.z, xm.w};
        const float rr[4] = {xr4.x, xr4.y, xr4.z, xr4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (j + e < p.n) {
                acc->xx = fmaf(vv[e], vv[e], acc->xx);
                if (p.criterion == 1) {
                    const float xr = rr[e];
                    const float dd = vv[e] - xr;
                    acc->e2 = fmaf(dd, dd, acc->e2);
                    acc->r2 = fmaf(xr, xr, acc->r2);
                }
            }
        }
    }
}

// Sum of rows [ga, gb) of column c of V (float4), in ascending gamma, with the
// loads issued in batches of B independent L2 reads.
template <int B>
__device__ __forceinline__ float4 sum_column(const KParams& p, int c, int ga, int gb) {
    const float* col = p.V + (size_t)c * 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int g0 = ga; g0 < gb; g0 += B) {
        float4 w[B];
#pragma unroll
        for (int u = 0; u < B; ++u)
            w[u] = (g0 + u < gb) ? ldcg4(col + (size_t)(g0 + u) * (size_t)p.ldv) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < B; ++u) {
            acc.x += w[u].x; acc.y += w[u].y; acc.z += w[u].z; acc.w += w[u].w;
        }
    }
    return acc;
}

// x <- x + (1/q) sum_gamma d_gamma (d_gamma = V[gamma]) for this CTA's
// contiguous slice of float4 columns; x is read from x0 in the first round and
// from xbuf afterwards (only the slice's owner reads and writes it here).
// When the slice is narrower than the CTA, the workers are split into
// `groups` contiguous ranges, each summed in ascending gamma by one thread, and
// the group sums are added in ascending group order: a fixed two-level order,
// the same on every run.  With chk, the thread's check partials of the stored
// columns are accumulated.
template <int NT>
__device__ __forceinline__ void average_slice(const KParams& p, float4* avg, bool first, ChkAcc* chk) {
    const int tid = threadIdx.x;
    const int n4 = p.n4;
    const int G = gridDim.x;
    const int cols = (n4 + G - 1) / G;
    const int c0 = blockIdx.x * cols;
    const int c1 = min(n4, c0 + cols);
    const int nc = c1 - c0;
    const float rq = 1.0f / (float)p.q;
    // loads in flight per thread: fewer where 512 consumers share the registers
    constexpr int kAvgBatch = NT >= 512 ? 8 : 16;
    if (nc <= 0) return;
    if (nc >= NT) {
        for (int c = c0 + tid; c < c1; c += NT) {
            const float4 xo = load_x_old(p, c, first);
            const float4 xr = load_xref(p, c, chk != nullptr);
            const float4 acc = sum_column<kAvgBatch>(p, c, 0, p.vrows);
            store_x(p, c, make_float4(fmaf(acc.x, rq, xo.x), fmaf(acc.y, rq, xo.y), fmaf(acc.z, rq, xo.z),
                                      fmaf(acc.w, rq, xo.w)), chk, xr);
        }
        return;
    }
    int groups = NT / nc;
    if (groups > p.vrows) groups = p.vrows;
    const int per = (p.vrows + groups - 1) / groups;
    const int cl = tid % nc, g = tid / nc;
    float4 xo = make_float4(0.f, 0.f, 0.f, 0.f), xr = xo;
    if (tid < nc) {
        xo = load_x_old(p, c0 + tid, first);
        xr = load_xref(p, c0 + tid, chk != nullptr);
    }
    if (g < groups) {
        const int ga = g * per, gb = min(p.vrows, ga + per);
        avg[g * nc + cl] = sum_column<kAvgBatch>(p, c0 + cl, ga, gb);
    }
    named_bar_sync(1, NT);
    if (tid < nc) {
        float4 acc = avg[tid];
        for (int gg = 1; gg < groups; ++gg) {
            const float4 w = avg[gg * nc + tid];
            acc.x += w.x; acc.y += w.y; acc.z += w.z; acc.w += w.w;
        }
        store_x(p, c0 + tid, make_float4(fmaf(acc.x, rq, xo.x), fmaf(acc.y, rq, xo.y), fmaf(acc.z, rq, xo.z),
                                         fmaf(acc.w, rq, xo.w)), chk, xr);
    }
}

// CTA sum of the threads' check partials in a fixed order (warp butterfly, then
// warps in ascending order), published by thread 0 as this CTA's entry of
// p.chkpart before the grid barrier that follows.  In two halves around a CTA
// barrier the caller may already have: the warp sums into shared memory, then
// thread 0's sum over the warps.
template <int NT>
__device__ __forceinline__ void check_warp_partials(ChkAcc a, double* chk) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* sh = reinterpret_cast<float*>(chk);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a.xx += __shfl_xor_sync(0xffffffffu, a.xx, o);
        a.e2 += __shfl_xor_sync(0xffffffffu, a.e2, o);
        a.r2 += __shfl_xor_sync(0xffffffffu, a.r2, o);
    }
    if (lane == 0) {
        sh[warp] = a.xx;
        sh[32 + warp] = a.e2;
        sh[64 + warp] = a.r2;
    }
}

template <int NT>
__device__ __forceinline__ void check_cta_partial(const KParams& p, const double* chk) {
    constexpr int NW = NT / 32;
    const float* sh = reinterpret_cast<const float*>(chk);
    float xx = 0.f, e2 = 0.f, r2 = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        xx += sh[w];
        e2 += sh[32 + w];
        r2 += sh[64 + w];
    }
    reinterpret_cast<float4*>(p.chkpart)[blockIdx.x] = make_float4(xx, e2, r2, 0.f);
}

template <int NT>
__device__ __forceinline__ void publish_check(const KParams& p, ChkAcc a, double* chk) {
    check_warp_partials<NT>(a, chk);
    named_bar_sync(1, NT);
    if (threadIdx.x == 0) check_cta_partial<NT>(p, chk);
}

// Totals of all CTAs' check partials, summed by warp 0 in a fixed order (lane l
// takes CTAs l, l + 32, ... in ascending order, then a butterfly): every CTA
// computes the same values from the same data.  Result in chk[0..2] for the
// whole CTA after the closing barrier.
template <int NT>
__device__ __forceinline__ void combine_check(const KParams& p, double* chk) {
    if ((threadIdx.x >> 5) == 0) {
        const int lane = threadIdx.x & 31;
        const int G = (int)gridDim.x;
        float4 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int g = lane + 32 * u;
            w[u] = g < G ? __ldcg(reinterpret_cast<const float4*>(p.chkpart) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float xx = 0.f, e2 = 0.f, r2 = 0.f;
        for (int u = 0; u < 8; ++u) {
            xx += w[u].x;
            e2 += w[u].y;
            r2 += w[u].z;
        }
        for (int g = lane + 256; g < G; g += 32) {   // grids beyond 256 CTAs
            const float4 t = __ldcg(reinterpret_cast<const float4*>(p.chkpart) + g);
            xx += t.x;
            e2 += t.y;
            r2 += t.z;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            xx += __shfl_xor_sync(0xffffffffu, xx, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
            r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        }
        if (lane == 0) {
            float* sh = reinterpret_cast<float*>(chk);
            sh[0] = xx;
            sh[1] = e2;
            sh[2] = r2;
        }
    }
    named_bar_sync(1, NT);
}

// Shared memory after the stages: avg[NT] float4, full[S] + empty[S] mbarriers,
// meta[S] float4, red[2][16][32] float (warp partials, double-buffered), chk[96]
// double, pbuf[32] float4 (the producer's batch of draws), Ctrl.
constexpr int kRedSlots = 16;   // partial sums reduced per group of rows (W + W(W-1)/2)
__host__ __device__ inline size_t solve_ctrl_bytes(int S, int nt) {
    return (size_t)nt * 16 + (size_t)S * 32 + 2 * kRedSlots * 32 * 4 + 96 * 8 + 32 * 16 + 64;
}

// Rows of one look-ahead group (W > 1): the consumers take W consecutive rows
// q_0 .. q_{W-1} of their stream (stored values; A_r = s_r q_r with s_r the FP8
// row scale, 1 otherwise) and, from the same v = x + d, form in one pass
//   g_r = <q_r, v>   and   G_rl = <q_r, q_l>  (l < r),
// reduce these W + W(W-1)/2 sums across the CTA once, then resolve the
// coefficients of the sequential projections with the scalar recurrence
//   h_r = g_r + sum_{l<r} c_l G_rl   (= <q_r, v after projections 0 .. r-1>)
//   c_r = omega (b_r - s_r h_r) / ||A_r||^2 * s_r,
// and apply d += sum_r c_r q_r.  In exact arithmetic this is the same as W
// projections of Eq. (alg) one after the other; it pays the CTA-wide reduction
// once per W rows instead of once per row.
template <int W>
struct GroupIdx {
    static constexpr int NV = W + W * (W - 1) / 2;
    __device__ static constexpr int gram(int r, int l) { return W + r * (r - 1) / 2 + l; }
};

// MINB = CTAs per SM the variant is built for (its register budget): 2 lets the
// grid hold two workers per SM (more workers per round, smaller per-CTA share).
// JAC = the CTA sums independent single projections from the round's x (RKA with
// the workers spread over the CTAs, KParams::jacobi); W = 1 only.
template <int NT, int VPT, int ELT, bool KEEP_A, int W, int MINB = 1, bool JAC = false, bool XS = false>
__global__ void __launch_bounds__(NT + 32, MINB) rkab_kernel(const KParams p) {
    static_assert(!JAC || W == 1, "independent projections are not grouped");
    static_assert(W == 1 || !KEEP_A, "look-ahead groups re-read their rows");
    static_assert(!XS || (KEEP_A && W == 1), "x in shared memory only with the fused pass");
    static_assert(GroupIdx<W>::NV <= kRedSlots, "too many partial sums per group");
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int NW = NT / 32;
    const int S = p.stages;
    uint8_t* stages = smem;
    // XS: the round's start point x lives in shared memory after the stages, each
    // thread's slices at the same indices as in registers (only that thread reads
    // and writes them, so no barrier guards them); the registers it frees hold the
    // widened row between the dot and the update
    float4* xs = reinterpret_cast<float4*>(smem + (size_t)S * p.stage_stride);  // [NT * VPT] if XS
    float4* avg = xs + (XS ? NT * VPT : 0);                                     // [NT]
    uint64_t* full = reinterpret_cast<uint64_t*>(avg + NT);
    uint64_t* empty = full + S;
    float4* meta = reinterpret_cast<float4*>(empty + S);
    float* red = reinterpret_cast<float*>(meta + S);          // [2][kRedSlots][32] partials
    double* chk = reinterpret_cast<double*>(red + 2 * kRedSlots * 32);  // [3][32] check partials
    float4* pbuf = reinterpret_cast<float4*>(chk + 96);                  // [32] producer batch
    volatile Ctrl* ctrl = reinterpret_cast<volatile Ctrl*>(pbuf + 32);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t alpha_c = cta_projections<JAC>(p);   // projections per round in this CTA
    const int64_t total = p.rounds * alpha_c;
    constexpr bool jac = JAC;                     // dots from the round's x only
    int* status = &p.info->status;

    {
        uint4* z = reinterpret_cast<uint4*>(stages);
        const size_t nz = (size_t)S * p.stage_stride / 16;
        for (size_t i = tid; i < nz; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    // the zeros must be visible to the bulk copies' async proxy before any copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
    // the cyclic sweep visits every row, also those whose ||A_i||^2 lies outside the
    // float32 range of the projection (never drawn by the random selections)
    if (p.sampling == RK_SAMPLE_CYCLIC && p.setup->range_rows != 0) {
        if (tid == 0) set_status(status, RK_EINVAL);
        return;
    }
    if (warp == NW) {
        producer_loop<ELT, JAC>(p, stages, full, empty, meta, ctrl, pbuf);
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
        if constexpr (XS) xs[idx] = t;
        else v[k] = t;
        d[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    const int rem = p.n & 3;
    int tail_k = -1;
    if (rem && ((n4 - 1 - tid) % NT) == 0 && n4 - 1 >= tid) tail_k = (n4 - 1 - tid) / NT;
    int s = 0;
    uint32_t ph = 0;
    int rp = 0;
    int64_t t = 0;
    bool ok = true;
    float* Vg = p.V + (size_t)gamma * (size_t)p.ldv;
    for (int64_t r = 0; r < p.rounds && ok; ++r) {
      if constexpr (W > 1) {
        constexpr int NV = GroupIdx<W>::NV;
        for (int64_t j = 0; j < alpha_c; j += W) {
            const int wc = (alpha_c - j) < W ? (int)(alpha_c - j) : W;
            int sg[W];
            uint32_t pg[W];
            bool got = true;
#pragma unroll
            for (int rr = 0; rr < W; ++rr) {
                const int sr = s + rr;
                sg[rr] = sr >= p.stages ? sr - p.stages : sr;
                pg[rr] = sr >= p.stages ? (ph ^ 1u) : ph;
                if (rr < wc) got = wait_parity(&full[sg[rr]], pg[rr], p.timeout_ns, status) && got;
            }
            float acc[NV];
#pragma unroll
            for (int u = 0; u < NV; ++u) acc[u] = 0.f;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int idx = tid + k * NT;
                float4 aq[W];
#pragma unroll
                for (int rr = 0; rr < W; ++rr) {
                    aq[rr] = rr < wc ? slice<ELT>(stages + (size_t)sg[rr] * p.stage_stride, idx, k, tail_k, rem)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int rr = 0; rr < W; ++rr) {
                    float g = acc[rr];
                    g = fmaf(aq[rr].x, v[k].x, g);
                    g = fmaf(aq[rr].y, v[k].y, g);
                    g = fmaf(aq[rr].z, v[k].z, g);
                    g = fmaf(aq[rr].w, v[k].w, g);
                    g = fmaf(aq[rr].x, d[k].x, g);
                    g = fmaf(aq[rr].y, d[k].y, g);
                    g = fmaf(aq[rr].z, d[k].z, g);
                    g = fmaf(aq[rr].w, d[k].w, g);
                    acc[rr] = g;
#pragma unroll
                    for (int ll = 0; ll < rr; ++ll) {
                        float h = acc[GroupIdx<W>::gram(rr, ll)];
                        h = fmaf(aq[rr].x, aq[ll].x, h);
                        h = fmaf(aq[rr].y, aq[ll].y, h);
                        h = fmaf(aq[rr].z, aq[ll].z, h);
                        h = fmaf(aq[rr].w, aq[ll].w, h);
                        acc[GroupIdx<W>::gram(rr, ll)] = h;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < NV; ++u) {
#pragma unroll
                for (int o = 16; o; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
            }
            if (lane == 0) {
#pragma unroll
                for (int u = 0; u < NV; ++u) red[(rp * kRedSlots + u) * 32 + warp] = acc[u];
            }
            if (!bar_and(1, NT, got)) { ok = false; break; }
            float tot[NV];
#pragma unroll
            for (int u = 0; u < NV; ++u) {
                tot[u] = cta_sum<NW>(red + (rp * kRedSlots + u) * 32);
            }
            rp ^= 1;
            float c[W];
#pragma unroll
            for (int rr = 0; rr < W; ++rr) {
                c[rr] = 0.f;
                if (rr < wc) {
                    float h = tot[rr];
#pragma unroll
                    for (int ll = 0; ll < rr; ++ll) h = fmaf(c[ll], tot[GroupIdx<W>::gram(rr, ll)], h);
                    const float4 mb = meta[sg[rr]];   // b_r, 1/||A_r||^2, row scale s_r
                    c[rr] = p.omega * (mb.x - mb.z * h) * mb.y * mb.z;
                }
            }
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int idx = tid + k * NT;
#pragma unroll
                for (int rr = 0; rr < W; ++rr) {
                    if (rr < wc) {
                        const float4 aq = slice<ELT>(stages + (size_t)sg[rr] * p.stage_stride, idx, k, tail_k, rem);
                        d[k].x = fmaf(c[rr], aq.x, d[k].x);
                        d[k].y = fmaf(c[rr], aq.y, d[k].y);
                        d[k].z = fmaf(c[rr], aq.z, d[k].z);
                        d[k].w = fmaf(c[rr], aq.w, d[k].w);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
#pragma unroll
                for (int rr = 0; rr < W; ++rr) {
                    if (rr < wc) mbar_arrive(&empty[sg[rr]]);
                }
            }
            s += wc;
            if (s >= p.stages) { s -= p.stages; ph ^= 1u; }
            t += wc;
        }
      } else if constexpr (KEEP_A) {
        // One pass over the slices per row: the update of row t-1 (kept in
        // registers with its coefficient) is applied in the pass that forms the
        // dot of row t, then row t replaces it; the last update of the round is
        // applied before the average.
        float4 a[VPT];
        float cprev = 0.f;
#pragma unroll
        for (int k = 0; k < VPT; ++k) a[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t j = 0; j < alpha_c; ++j, ++t) {
            const bool got = wait_parity(&full[s], ph, p.timeout_ns, status);
            const uint8_t* stg = stages + (size_t)s * p.stage_stride;
            const float4 mb = meta[s];   // b_i, 1/||A_i||^2, row scale
            // two packed accumulators (elements x,y and z,w of the slices); each
            // packed FMA is two independent float32 FMAs
            float2 p01 = make_float2(0.f, 0.f), p23 = make_float2(0.f, 0.f);
            const float2 cc = make_float2(cprev, cprev);
#define RK_FUSED_SLICE(LOADEXPR)                                                        \
            {                                                                           \
                const float4 ak = LOADEXPR;                                             \
                const float4 xk = XS ? xs[tid + k * NT] : v[k];                         \
                const float2 dlo = __ffma2_rn(cc, make_float2(a[k].x, a[k].y),          \
                                              make_float2(d[k].x, d[k].y));             \
                const float2 dhi = __ffma2_rn(cc, make_float2(a[k].z, a[k].w),          \
                                              make_float2(d[k].z, d[k].w));             \
                const float2 alo = make_float2(ak.x, ak.y), ahi = make_float2(ak.z, ak.w); \
                p01 = __ffma2_rn(alo, make_float2(xk.x, xk.y), p01);                    \
                p23 = __ffma2_rn(ahi, make_float2(xk.z, xk.w), p23);                    \
                if (!jac) {                                                             \
                    p01 = __ffma2_rn(alo, dlo, p01);                                    \
                    p23 = __ffma2_rn(ahi, dhi, p23);                                    \
                }                                                                       \
                d[k] = make_float4(dlo.x, dlo.y, dhi.x, dhi.y);                         \
                a[k] = ak;                                                              \
            }
            if (rem == 0) {
#pragma unroll
                for (int k = 0; k < VPT; ++k) RK_FUSED_SLICE(load4<ELT>(stg, tid + k * NT))
            } else {
#pragma unroll
                for (int k = 0; k < VPT; ++k) RK_FUSED_SLICE(slice<ELT>(stg, tid + k * NT, k, tail_k, rem))
            }
#undef RK_FUSED_SLICE
            __syncwarp();
            // a stage whose copy this warp did not see land is never released: the
            // producer must not refill it while that copy may still be writing
            if (lane == 0 && got) mbar_arrive(&empty[s]);
            float part = (p01.x + p01.y) + (p23.x + p23.y);
#pragma unroll
            for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) red[rp * kRedSlots * 32 + warp] = part;
            if (!bar_and(1, NT, got)) { ok = false; break; }
            // every thread sums the NW warp partials in the same order, so all
            // threads of the CTA hold the same dot
            const float dot = cta_sum<NW>(red + rp * kRedSlots * 32);
            rp ^= 1;
            // A_i = s_i q_i: <A_i, v> = s_i <q_i, v>, d += (scale s_i) q_i
            cprev = p.omega * (mb.x - mb.z * dot) * mb.y * mb.z;
            if (++s == p.stages) { s = 0; ph ^= 1u; }
        }
        {
            const float2 cc = make_float2(cprev, cprev);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const float2 dlo = __ffma2_rn(cc, make_float2(a[k].x, a[k].y), make_float2(d[k].x, d[k].y));
                const float2 dhi = __ffma2_rn(cc, make_float2(a[k].z, a[k].w), make_float2(d[k].z, d[k].w));
                d[k] = make_float4(dlo.x, dlo.y, dhi.x, dhi.y);
            }
        }
      } else {
        for (int64_t j = 0; j < alpha_c; ++j, ++t) {
            const bool got = wait_parity(&full[s], ph, p.timeout_ns, status);
            const uint8_t* stg = stages + (size_t)s * p.stage_stride;
            const float4 mb = meta[s];   // b_i, 1/||A_i||^2, row scale
            // four independent accumulators (one per element of a slice, two packed
            // pairs: one FFMA2 per two products) keep the FMA pipe fed; they are
            // combined in a fixed order
            float2 p01 = make_float2(0.f, 0.f), p23 = make_float2(0.f, 0.f);
            float4 a[KEEP_A ? VPT : 1];
            // the tail mask only when n is not a multiple of 4 (a uniform branch: the
            // loop without it has no per-slice compare and selects)
#define RK_DOT_LOOP(LOADEXPR)                                                           \
            _Pragma("unroll")                                                           \
            for (int k = 0; k < VPT; ++k) {                                             \
                const int idx = tid + k * NT;                                           \
                const float4 ak = LOADEXPR;                                             \
                if constexpr (KEEP_A) a[k] = ak;                                        \
                const float2 alo = make_float2(ak.x, ak.y), ahi = make_float2(ak.z, ak.w); \
                p01 = __ffma2_rn(alo, make_float2(v[k].x, v[k].y), p01);                \
                p23 = __ffma2_rn(ahi, make_float2(v[k].z, v[k].w), p23);                \
                if (!jac) {                                                             \
                    p01 = __ffma2_rn(alo, make_float2(d[k].x, d[k].y), p01);            \
                    p23 = __ffma2_rn(ahi, make_float2(d[k].z, d[k].w), p23);            \
                }                                                                       \
            }
            if (rem == 0) {
                RK_DOT_LOOP(load4<ELT>(stg, idx))
            } else {
                RK_DOT_LOOP(slice<ELT>(stg, idx, k, tail_k, rem))
            }
#undef RK_DOT_LOOP
            if constexpr (KEEP_A) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            float part = (p01.x + p01.y) + (p23.x + p23.y);
#pragma unroll
            for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) red[rp * kRedSlots * 32 + warp] = part;
            if (!bar_and(1, NT, got)) { ok = false; break; }
            // every thread sums the NW warp partials in the same order, so all
            // threads of the CTA hold the same dot
            const float dot = cta_sum<NW>(red + rp * kRedSlots * 32);
            rp ^= 1;
            // A_i = s_i q_i: <A_i, v> = s_i <q_i, v>, d += (scale s_i) q_i
            const float scale = p.omega * (mb.x - mb.z * dot) * mb.y * mb.z;
            const float2 sc2 = make_float2(scale, scale);
#define RK_UPD_LOOP(LOADEXPR)                                                           \
            _Pragma("unroll")                                                           \
            for (int k = 0; k < VPT; ++k) {                                             \
                const int idx = tid + k * NT;                                           \
                (void)idx;                                                              \
                float4 ak;                                                              \
                if constexpr (KEEP_A) ak = a[k];                                        \
                else ak = LOADEXPR;                                                     \
                const float2 dlo = __ffma2_rn(sc2, make_float2(ak.x, ak.y), make_float2(d[k].x, d[k].y)); \
                const float2 dhi = __ffma2_rn(sc2, make_float2(ak.z, ak.w), make_float2(d[k].z, d[k].w)); \
                d[k] = make_float4(dlo.x, dlo.y, dhi.x, dhi.y);                         \
            }
            if (rem == 0) {
                RK_UPD_LOOP(load4<ELT>(stg, idx))
            } else {
                RK_UPD_LOOP(slice<ELT>(stg, idx, k, tail_k, rem))
            }
#undef RK_UPD_LOOP
            if constexpr (!KEEP_A) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if (++s == p.stages) { s = 0; ph ^= 1u; }
        }
      }
        if (!ok) break;

        // ---- average: x <- x + (1/q) sum_gamma d_gamma ----
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int idx = tid + k * NT;
            if (idx < n4) reinterpret_cast<float4*>(Vg)[idx] = d[k];
        }
        named_bar_sync(1, NT);
        if (tid == 0) ctrl->flag = grid_sync(&p.info->bar_arrivals, 2ull * (unsigned long long)r, gridDim.x,
                                             status, p.timeout_ns) ? 1 : 0;
        named_bar_sync(1, NT);
        if (!ctrl->flag) { ok = false; break; }
        // ---- convergence / divergence check (identical in every CTA): each CTA
        // sums its own slice of the new x while averaging; the totals are formed
        // after the barrier from all CTAs' partials ----
        const int64_t done = r + 1;
        const bool last = (done == p.rounds);
        const bool check = p.check_every > 0 && (done % p.check_every == 0 || last);
        ChkAcc ca{0.f, 0.f, 0.f};
        average_slice<NT>(p, avg, r == 0, check ? &ca : nullptr);
        if (check) check_warp_partials<NT>(ca, chk);
        named_bar_sync(1, NT);
        if (check && tid == 0) check_cta_partial<NT>(p, chk);
        if (tid == 0) ctrl->flag = grid_sync(&p.info->bar_arrivals, 2ull * (unsigned long long)r + 1ull,
                                             gridDim.x, status, p.timeout_ns) ? 1 : 0;
        named_bar_sync(1, NT);
        if (!ctrl->flag) { ok = false; break; }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int idx = tid + k * NT;
            const float4 xn = (idx < n4) ? ldcg4(p.xbuf + (size_t)idx * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (XS) xs[idx] = xn;
            else v[k] = xn;
            d[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }

        if (check) {
            combine_check<NT>(p, chk);
            const float* sh = reinterpret_cast<const float*>(chk);
            const float XX = sh[0], E2 = sh[1], R2 = sh[2];
            named_bar_sync(1, NT);
            // float32 throughout: the float64 pipe of this device is slow, and
            // every thread takes the decision
            float mf = -1.f;
            if (p.criterion == 1) mf = (R2 > 0.f) ? sqrtf(E2 / R2) : sqrtf(E2);
            const double metric = (double)mf;
            const bool diverged = !isfinite(XX) || (p.criterion == 1 && !isfinite(mf));
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

typedef void (*SolveKernelFn)(const KParams);

struct SolveVariant {
    int nt, vpt;
    bool keep_a;
    int w;              // rows per look-ahead group
    SolveKernelFn fn;
    int minb;           // CTAs per SM the register budget allows (1 or 2)
    bool jac;           // independent projections from the round's x (RKA spread over CTAs)
    bool xs;            // x in shared memory (NT * VPT float4 after the stages)
};

// Instantiation tables (one translation unit per stored type).
const SolveVariant* solve_variants_f32(int* count);
const SolveVariant* solve_variants_bf16(int* count);
const SolveVariant* solve_variants_fp8(int* count);

}  // namespace rk
