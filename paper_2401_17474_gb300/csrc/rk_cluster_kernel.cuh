// rk_cluster_kernel.cuh -- RKAB with each worker spread over a thread-block
// cluster of C CTAs (Section 3.4.1 / Algorithm 3, same iteration as
// rk_solve_kernel.cuh).  Instantiated in rk_cluster_*.cu, launched by rk_solve.cu.
//
// Time to tolerance is the number of projections one worker makes in sequence
// times the latency of one projection; a worker on one SM is limited by the
// CTA-wide reduction each row needs.  Here a worker's row is split into C
// contiguous chunks of columns, one per CTA of its cluster: every CTA streams
// only its chunk of each sampled row (bulk copy into its own ring of stages),
// holds x and d for its chunk in registers, and the cluster resolves W rows at
// a time:
//   g_r = <q_r, v>,  G_rl = <q_r, q_l> (l < r)       partial sums over the chunk
//   reduce-scatter in each warp, warp totals in shared memory, CTA totals sent
//   to every CTA of the cluster (st.async + mbarrier transaction counts), summed
//   in rank order (identical in every CTA),
//   h_r = g_r + sum_{l<r} c_l G_rl,  c_r = omega (b_r - s_r h_r) / ||A_r||^2 s_r,
//   d += sum_r c_r q_r  over the chunk,
// which equals W projections of Eq. (alg) one after the other in exact
// arithmetic.  The averaging of the q workers and the grid barriers are those
// of the one-CTA kernel; the convergence check reads the whole averaged vector,
// so every CTA of the grid takes the same decision.
#pragma once

#include "rk_solve_kernel.cuh"

namespace rk {

constexpr int kClusterMax = 16;
constexpr int kNVP = 32;   // partial sums per group, padded: one per lane after the reduce-scatter

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared::cluster address of `local` (a shared address of this CTA) in CTA `rank`.
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

// Store one float into another CTA's shared memory and count 4 bytes on its mbarrier.
__device__ __forceinline__ void st_async_f32(uint32_t raddr, float v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
                 ::"r"(raddr), "r"(__float_as_uint(v)), "r"(rbar) : "memory");
}

// Warp reduce-scatter of 32 values per lane: afterwards lane u holds the sum
// over the warp of value u.  Five halving steps (offsets 16, 8, 4, 2, 1): a
// lane keeps the half of its current values selected by its lane bit and adds
// the partner's copy of that half; 31 shuffles in all.
__device__ __forceinline__ float reduce_scatter32(float (&v)[kNVP], int lane) {
#pragma unroll
    for (int o = 16, cnt = 32; o >= 1; o >>= 1, cnt >>= 1) {
        const int half = cnt >> 1;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

template <int W>
struct CGroup {
    static constexpr int NV = W + W * (W - 1) / 2;
    __device__ static constexpr int gram(int r, int l) { return W + r * (r - 1) / 2 + l; }
};

// Shared memory after the stages: avg[NT] float4, full[S] + empty[S] + recv[2]
// mbarriers, meta[S] float4, wred[NW][32] float, recv buffers [2][16][32] float,
// chk[96] double, pbuf[32] float4, Ctrl.
__host__ __device__ inline size_t cluster_ctrl_bytes(int S, int nt) {
    return (size_t)nt * 16 + (size_t)S * 32 + 16 + (size_t)(nt / 32) * kNVP * 4 +
           2 * kClusterMax * kNVP * 4 + 96 * 8 + 32 * 16 + 64;
}

struct CParams {
    KParams k;          // row source, tables, iterate buffers, options (chunk-local copy sizes)
    int chunk;          // slices per CTA (multiple of 4)
};

// Thread 0, once every CTA of the cluster has stopped sending: wait (bounded) for the
// receive buffer it armed last if it never saw that group's totals land.  Kept out of
// line: it runs once a launch, and the solve loop's registers are not its concern.
static __device__ __noinline__ void cluster_drain_receive(uint64_t* recvbar, volatile Ctrl* ctrl, uint64_t timeout_ns,
                                                   int* status) {
    const int pw = ctrl->pad;
    if (pw & 4) wait_parity(&recvbar[pw & 1], (uint32_t)((pw >> 1) & 1), drain_limit_ns(timeout_ns), status);
}

template <int NT, int VPT, int ELT, int W>
__global__ void __launch_bounds__(NT + 32, 1) rkab_cluster_kernel(const CParams cp) {
    static_assert(CGroup<W>::NV <= kNVP, "too many partial sums per group");
    const KParams& p = cp.k;
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int NW = NT / 32;
    const int S = p.stages;
    uint8_t* stages = smem;
    float4* avg = reinterpret_cast<float4*>(smem + (size_t)S * p.stage_stride);  // [NT]
    uint64_t* full = reinterpret_cast<uint64_t*>(avg + NT);
    uint64_t* empty = full + S;
    uint64_t* recvbar = empty + S;                                       // [2]
    float4* meta = reinterpret_cast<float4*>(recvbar + 2);
    float* wred = reinterpret_cast<float*>(meta + S);                   // [NW][32]
    float* recv = wred + NW * kNVP;                                     // [2][16][32]
    double* chk = reinterpret_cast<double*>(recv + 2 * kClusterMax * kNVP);
    float4* pbuf = reinterpret_cast<float4*>(chk + 96);
    volatile Ctrl* ctrl = reinterpret_cast<volatile Ctrl*>(pbuf + 32);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t total = p.rounds * p.alpha;
    int* status = &p.info->status;
    const uint32_t crank = cluster_ctarank();
    const uint32_t csize = cluster_nctarank();

    {
        uint4* z = reinterpret_cast<uint4*>(stages);
        const size_t nz = (size_t)S * p.stage_stride / 16;
        for (size_t i = tid; i < nz; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        mbar_init(&recvbar[0], 1);
        mbar_init(&recvbar[1], 1);
        ctrl->stop_t = total;
        ctrl->flag = 0;
        ctrl->pad = 0;   // here: the receive buffer armed and not yet seen complete (4 | parity << 1 | buffer)
        fence_barrier_init();
    }
    __syncthreads();
    // every CTA of the cluster has its barriers ready before anyone sends to it
    cluster_sync_all();
    // a failed plan, or a cyclic sweep over rows the float32 projection cannot take
    const bool cyc_bad = p.sampling == RK_SAMPLE_CYCLIC && p.setup->range_rows != 0;
    const bool setup_ok = p.setup->status == 0 && !cyc_bad;
    if (!setup_ok && tid == 0) set_status(status, cyc_bad ? RK_EINVAL : RK_ESETUP);

    // this CTA's chunk of every row: slices [c0, c0 + nl)
    const int c0 = (int)crank * cp.chunk;
    const int nl = max(0, min(p.n4 - c0, cp.chunk));
    const int gamma = blockIdx.x / (int)csize;

    if (setup_ok && warp == NW) {
        // producer: the chunk's bytes of each row (the same draws in every CTA of the cluster)
        // this CTA copies slices [c0, c0 + nl) of each row: nl * 4 elements rounded up to
        // 16 bytes, which ends inside the row's lda extent (c0 is a multiple of 4 slices)
        constexpr uint32_t eb = ELT == ELT_F32 ? 4u : (ELT == ELT_BF16 ? 2u : 1u);
        const uint8_t* Ac = p.A + (size_t)c0 * 4 * eb;
        const uint32_t my_bytes = ((uint32_t)nl * 4u * eb + 15u) & ~15u;
        const int lane_ = lane;
        const int S_ = S;
        const int64_t total_ = total;
        const uint32_t worker = p.same_stream ? 0u : (uint32_t)gamma;
        const float ww = p.worker_weight ? __ldg(p.worker_weight + gamma) : 1.f;   // per-worker weight
        const uint64_t tbase = (uint64_t)p.round0 * (uint64_t)p.alpha;
        const uint64_t pol = policy_evict_first();
        int64_t issued = 0;
        int s = 0;
        uint32_t pass = 0;
        bool stop = false;
        for (int64_t base = 0; base < total_ && !stop; base += 32) {
            const int64_t tl = base + lane_;
            if (tl < total_) {
                uint32_t row = draw_row(p, worker, tbase + (uint64_t)tl);
                if (row >= p.m) {   // a row block of zero weight: nothing to draw
                    set_status(status, RK_EINVAL);
                    row = 0;
                }
                const float sc = (ELT == ELT_FP8) ? __ldg(p.row_scale + row) : 1.f;
                const float wi = p.row_weight ? __ldg(p.row_weight + row) : 1.f;
                pbuf[lane_] = make_float4(__uint_as_float(row), __ldg(p.b + row), __ldg(p.inv + row) * wi * ww, sc);
            }
            __syncwarp();
            if (lane_ == 0) {
                const int64_t rem_ = total_ - base;
                const int cnt = rem_ < 32 ? (int)rem_ : 32;
                for (int k = 0; k < cnt && !stop; ++k) {
                    const int64_t tt = base + k;
                    if (tt >= ctrl->stop_t) { stop = true; break; }
                    if (tt >= S_) {
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
                    mbar_arrive_expect_tx(&full[s], my_bytes);
                    if (my_bytes)
                        bulk_g2s(stages + (size_t)s * p.stage_stride, Ac + (size_t)row * (size_t)p.lda_bytes,
                                 my_bytes, &full[s], pol);
                    issued = tt + 1;
                    if (++s == S_) { s = 0; pass ^= 1u; }
                }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            __syncwarp();
        }
        if (lane_ == 0) {
            const int64_t first = issued > S_ ? issued - S_ : 0;
            for (int64_t tt = first; tt < issued; ++tt) {
                const int st = (int)(tt % S_);
                const uint32_t par = (uint32_t)((tt / S_) & 1);
                wait_parity(&full[st], par, drain_limit_ns(p.timeout_ns), status);
            }
        }
        __syncwarp();
    } else if (setup_ok) {
        // ---------------- consumers ----------------
        constexpr int NV = CGroup<W>::NV;
        float4 v[VPT];
        float4 d[VPT];
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int li = tid + k * NT;
            float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (li < nl) {
                const int j = (c0 + li) * 4;
                t4.x = __ldg(p.x0 + j);
                if (j + 1 < p.n) t4.y = __ldg(p.x0 + j + 1);
                if (j + 2 < p.n) t4.z = __ldg(p.x0 + j + 2);
                if (j + 3 < p.n) t4.w = __ldg(p.x0 + j + 3);
            }
            v[k] = t4;
            d[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // the row's last slice lies in the CTA that owns slice n4 - 1
        const int rem = p.n & 3;
        int tail_k = -1;
        {
            const int li = p.n4 - 1 - c0;
            if (rem && li >= 0 && li < nl && (li - tid) >= 0 && ((li - tid) % NT) == 0) tail_k = (li - tid) / NT;
        }
        const uint32_t recv_local = smem_addr(recv);
        const uint32_t recvbar_local = smem_addr(recvbar);
        int s = 0;
        uint32_t ph = 0;
        int64_t t = 0;
        int64_t grp = 0;   // groups resolved so far (double-buffer index and phase)
        bool ok = true;
        float* Vg = p.V + (size_t)gamma * (size_t)p.ldv + (size_t)c0 * 4;
        for (int64_t r = 0; r < p.rounds && ok; ++r) {
            for (int64_t j = 0; j < p.alpha; j += W) {
                const int wc = (p.alpha - j) < W ? (int)(p.alpha - j) : W;
                const int buf = (int)(grp & 1);
                const uint32_t rpar = (uint32_t)((grp >> 1) & 1);
                if (tid == 0) {
                    mbar_arrive_expect_tx(&recvbar[buf], csize * NV * 4u);
                    ctrl->pad = 4 | (int)(rpar << 1) | buf;
                }
                int sg[W];
                bool got = true;
#pragma unroll
                for (int rr = 0; rr < W; ++rr) {
                    const int sr = s + rr;
                    sg[rr] = sr >= S ? sr - S : sr;
                    const uint32_t pr = sr >= S ? (ph ^ 1u) : ph;
                    if (rr < wc) got = wait_parity(&full[sg[rr]], pr, p.timeout_ns, status) && got;
                }
                // packed accumulators: element pairs (x,y) and (z,w) of the slices are
                // accumulated separately and folded before the reduction
                float2 acc2[NV];
#pragma unroll
                for (int u = 0; u < NV; ++u) acc2[u] = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < VPT; ++k) {
                    float2 alo[W], ahi[W];
#pragma unroll
                    for (int rr = 0; rr < W; ++rr) {
                        const float4 aq = rr < wc ? slice<ELT>(stages + (size_t)sg[rr] * p.stage_stride, tid + k * NT, k, tail_k, rem)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                        alo[rr] = make_float2(aq.x, aq.y);
                        ahi[rr] = make_float2(aq.z, aq.w);
                    }
                    const float2 vlo = make_float2(v[k].x, v[k].y), vhi = make_float2(v[k].z, v[k].w);
                    const float2 dlo = make_float2(d[k].x, d[k].y), dhi = make_float2(d[k].z, d[k].w);
#pragma unroll
                    for (int rr = 0; rr < W; ++rr) {
                        float2 g = acc2[rr];
                        g = __ffma2_rn(alo[rr], vlo, g);
                        g = __ffma2_rn(ahi[rr], vhi, g);
                        g = __ffma2_rn(alo[rr], dlo, g);
                        g = __ffma2_rn(ahi[rr], dhi, g);
                        acc2[rr] = g;
#pragma unroll
                        for (int ll = 0; ll < rr; ++ll) {
                            float2 h = acc2[CGroup<W>::gram(rr, ll)];
                            h = __ffma2_rn(alo[rr], alo[ll], h);
                            h = __ffma2_rn(ahi[rr], ahi[ll], h);
                            acc2[CGroup<W>::gram(rr, ll)] = h;
                        }
                    }
                }
                float acc[kNVP];
#pragma unroll
                for (int u = 0; u < kNVP; ++u) acc[u] = u < NV ? acc2[u].x + acc2[u].y : 0.f;
                // warp totals: lane u holds partial sum u of this warp
                const float mine = reduce_scatter32(acc, lane);
                wred[warp * kNVP + lane] = mine;
                if (!bar_and(1, NT, got)) { ok = false; break; }
                // CTA totals (warp 0, lane u) sent to every CTA of the cluster, slot [crank][u]
                if (warp == 0 && lane < NV) {
                    float tot = 0.f;
#pragma unroll
                    for (int w = 0; w < NW; ++w) tot += wred[w * kNVP + lane];
                    const uint32_t slot = recv_local + (uint32_t)((buf * kClusterMax + (int)crank) * kNVP + lane) * 4u;
                    const uint32_t bar_l = recvbar_local + (uint32_t)buf * 8u;
                    for (uint32_t dst = 0; dst < csize; ++dst)
                        st_async_f32(map_rank(slot, dst), tot, map_rank(bar_l, dst));
                }
                // wait for all CTAs' totals of this group, then sum them in rank order
                if (!wait_parity(&recvbar[buf], rpar, p.timeout_ns, status)) got = false;
                else if (tid == 0) ctrl->pad = 0;
                float mytot = 0.f;
                if (lane < NV) {
                    for (uint32_t c = 0; c < csize; ++c) mytot += recv[(buf * kClusterMax + (int)c) * kNVP + lane];
                }
                float tv[NV];
#pragma unroll
                for (int u = 0; u < NV; ++u) tv[u] = __shfl_sync(0xffffffffu, mytot, u);
                float c[W];
#pragma unroll
                for (int rr = 0; rr < W; ++rr) {
                    c[rr] = 0.f;
                    if (rr < wc) {
                        float h = tv[rr];
#pragma unroll
                        for (int ll = 0; ll < rr; ++ll) h = fmaf(c[ll], tv[CGroup<W>::gram(rr, ll)], h);
                        const float4 mb = meta[sg[rr]];
                        c[rr] = p.omega * (mb.x - mb.z * h) * mb.y * mb.z;
                    }
                }
#pragma unroll
                for (int k = 0; k < VPT; ++k) {
                    float2 dlo = make_float2(d[k].x, d[k].y), dhi = make_float2(d[k].z, d[k].w);
#pragma unroll
                    for (int rr = 0; rr < W; ++rr) {
                        if (rr < wc) {
                            const float4 aq = slice<ELT>(stages + (size_t)sg[rr] * p.stage_stride, tid + k * NT, k, tail_k, rem);
                            const float2 cc = make_float2(c[rr], c[rr]);
                            dlo = __ffma2_rn(cc, make_float2(aq.x, aq.y), dlo);
                            dhi = __ffma2_rn(cc, make_float2(aq.z, aq.w), dhi);
                        }
                    }
                    d[k] = make_float4(dlo.x, dlo.y, dhi.x, dhi.y);
                }
                __syncwarp();
                if (lane == 0) {
#pragma unroll
                    for (int rr = 0; rr < W; ++rr) {
                        if (rr < wc) mbar_arrive(&empty[sg[rr]]);
                    }
                }
                // the wred slots are rewritten next group only after this barrier
                if (!bar_and(1, NT, got)) { ok = false; break; }
                s += wc;
                if (s >= S) { s -= S; ph ^= 1u; }
                t += wc;
                ++grp;
            }
            if (!ok) break;

            // ---- average: x <- x + (1/q) sum_gamma d_gamma (column slices over the grid) ----
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int li = tid + k * NT;
                if (li < nl) reinterpret_cast<float4*>(Vg)[li] = d[k];
            }
            named_bar_sync(1, NT);
            if (tid == 0) ctrl->flag = grid_sync(&p.info->bar_arrivals, 2ull * (unsigned long long)r,
                                                 gridDim.x, status, p.timeout_ns) ? 1 : 0;
            named_bar_sync(1, NT);
            if (!ctrl->flag) { ok = false; break; }
            // ---- convergence / divergence check over the whole averaged vector:
            // partials of each CTA's slice while averaging, totals after the barrier ----
            const int64_t done = r + 1;
            const bool last = (done == p.rounds);
            const bool check = p.check_every > 0 && (done % p.check_every == 0 || last);
            ChkAcc ca{0.f, 0.f, 0.f};
            average_slice<NT>(p, avg, r == 0, check ? &ca : nullptr);
            named_bar_sync(1, NT);
            if (check) publish_check<NT>(p, ca, chk);
            if (tid == 0) ctrl->flag = grid_sync(&p.info->bar_arrivals, 2ull * (unsigned long long)r + 1ull,
                                                 gridDim.x, status, p.timeout_ns) ? 1 : 0;
            named_bar_sync(1, NT);
            if (!ctrl->flag) { ok = false; break; }
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int li = tid + k * NT;
                v[k] = (li < nl) ? ldcg4(p.xbuf + (size_t)(c0 + li) * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
                d[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }

            if (check) {
                combine_check<NT>(p, chk);
                const float* sh = reinterpret_cast<const float*>(chk);
                const float XX = sh[0], E2 = sh[1], R2 = sh[2];
                named_bar_sync(1, NT);
                float mf = -1.f;
                if (p.criterion == 1) mf = (R2 > 0.f) ? sqrtf(E2 / R2) : sqrtf(E2);
                const double metric = (double)mf;
                const bool diverged = !isfinite(XX) || (p.criterion == 1 && !isfinite(mf));
                if (blockIdx.x == 0 && tid == 0) {
                    p.info->rounds_done = done;
                    p.info->last_metric = metric;
                }
                if (diverged) {
                    if (tid == 0) set_status(status, RK_EDIVERGED);
                    ok = false;
                } else if (p.criterion == 1 && p.tol > 0.0 && metric < p.tol) {
                    break;  // converged: identical decision in every CTA of the grid
                }
            } else if (blockIdx.x == 0 && tid == 0) {
                p.info->rounds_done = done;
            }
        }
        if (tid == 0) ctrl->stop_t = t;
    }
    // no CTA of the cluster leaves while another may still write to its shared memory:
    // once every CTA has stopped sending (the first cluster barrier), a receive buffer
    // armed for a group whose totals did not all arrive (a wait that ran out) is waited
    // for again, bounded, so that every total already sent has landed before the second
    // barrier lets the CTAs go
    __syncwarp();
    cluster_sync_all();
    if (tid == 0) cluster_drain_receive(recvbar, ctrl, p.timeout_ns, status);
    cluster_sync_all();
}

typedef void (*ClusterKernelFn)(const CParams);

struct ClusterVariant {
    int nt, vpt, w;
    ClusterKernelFn fn;
};

const ClusterVariant* cluster_variants_f32(int* count);
const ClusterVariant* cluster_variants_bf16(int* count);
const ClusterVariant* cluster_variants_fp8(int* count);

}  // namespace rk
