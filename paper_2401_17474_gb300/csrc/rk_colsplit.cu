// rk_colsplit.cu -- RKA (alpha = 1; Algorithm 1, Eq. (rka_uni_weights), Eq. (rka_eq))
// with the columns of x split across the grid, for rows too long for one CTA's
// shared memory (the rows of A^T in the adjoint's minimum-norm solve, 200 KB to
// 800 KB): every one of the G CTAs (one per SM) owns a contiguous chunk of x's
// columns and, each round, streams that chunk of all q sampled rows.
//
// Round k, in every CTA g:
//   1. partial dots p_j^g = <A_j[chunk g], x[chunk g]> of the q rows j (the
//      round's draws of workers 0 .. q-1, the same draws as the one-CTA kernels:
//      worker j's projection counter is the round index), warp w forming rows
//      w, w + 8, ... whole over the chunk (x's chunk is held in shared memory);
//   2. the q partials go to global memory (double-buffered by round parity), one
//      grid barrier;
//   3. every CTA sums the G partials of each row in the same fixed order,
//      <A_j, x> = sum_g p_j^g, and forms c_j = omega w_j (b_j - <A_j, x>) / ||A_j||^2;
//   4. d = sum_j c_j A_j[chunk g], x[chunk g] += d / q: the average of the q
//      projections of Eq. (rka_uni_weights), held in the difference form (for chunks
//      of at most 128 slices each warp sums its own rows and the warp sums are added
//      in a fixed order; beyond, each thread sums its slices over all rows).
// A stage is released in step 4 as soon as its readers are done with it (the warp
// that owns the row, or every warp after each step of eight rows), so the ring holds
// at least the round's q rows; the producer fills the rest with the next round's rows.
// Checks (criterion, divergence) add a second grid barrier on the rounds they run.
#include "rk_solve_kernel.cuh"

namespace rk {

constexpr int kCsMaxQ = 64;    // workers a round (colsplit_fits in rk_internal.h)
constexpr int kCsSpare = 8;    // ring stages beyond two rounds' rows
constexpr int kCsProd = 4;     // producer warps (the ring's stage count is a multiple)
constexpr int kCsWarpRowsL = 4;   // slices a lane in the warp-rows update (chunks <= 128 slices)
constexpr int kCsSlicesAThread = 4;   // slices a thread in the rows-outer update (chunks <= 4 NT)

struct CSParams {
    KParams k;
    int chunk;          // slices (4 elements) of x per CTA, a multiple of 4
    int warp_rows;      // 1: the update takes a warp's own rows (chunks of at most
                        // kCsWarpRowsL * 32 slices); 0: a thread's slices over all rows
    float* part;        // [2][G][kCsMaxQ] partial dots (round parity, CTA, worker)
};

// Shared memory after the stages: full[S] + empty[S] mbarriers, meta[S] float4,
// xs[XP] float4 (this CTA's chunk of x, XP = chunk rounded up to 32 slices),
// dpart[NW][chunk] float4 (the update's warp sums, warp-rows mode only), grp[NT / 16][16]
// float4 (partial sums of the grid reduction), rowc[kCsMaxQ] float2 (c_j and row j's
// stage offset), chk[96] double, pbuf[kCsProd][32] float4, Ctrl (16 bytes), fillpar[S]
// bytes (the parity of each stage's last fill, for the producers' drain).
__host__ __device__ inline size_t cs_ctrl_bytes(int S, int nt, int chunk, bool warp_rows) {
    const size_t xp = (size_t)(chunk + 31) / 32 * 32;
    return (size_t)S * 32 + xp * 16 + (warp_rows ? (size_t)(nt / 32) * chunk * 16 : 0) + (size_t)nt * 16 + kCsMaxQ * 8 +
           96 * 8 + kCsProd * 32 * 16 + 16 + ((size_t)S + 15) / 16 * 16 + 64;
}

// Bytes of this CTA's chunk of a row: nl slices of 4 elements, rounded up to 16 bytes
// (which stays inside the row's lda extent: chunks start at multiples of 4 slices).
template <int ELT>
__device__ __forceinline__ uint32_t cs_copy_bytes(int nl) {
    constexpr uint32_t eb = ELT == ELT_F32 ? 4u : (ELT == ELT_BF16 ? 2u : 1u);
    return ((uint32_t)nl * 4u * eb + 15u) & ~15u;
}

// Non-blocking test of an mbarrier phase (mbarrier.test_wait: returns at once).
__device__ __forceinline__ bool cs_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Producer warps: rows of the q workers, round after round, into the ring (this
// CTA's chunk of each row).  Sequence index u = round * q + j uses stage u mod S.
// kCsProd warps share the rows: warp pw takes u = pw, pw + kCsProd, ... in order; S is
// a multiple of kCsProd, so a stage is always filled by the same warp and its empty
// barrier is at most one phase behind that warp's next use (the parity wait stays
// unambiguous).  A warp draws 32 of its rows at once; then for each row a lane writes
// the row's b_i, 1/||A_i||^2 and scale, arms the stage's full barrier with the chunk's
// byte count and issues one bulk copy of the chunk (the barrier's phase completes when
// the bytes have landed), and records the fill's parity in fillpar[stage].
template <int ELT>
__device__ void cs_producer(const CSParams& cp, uint8_t* stages, uint64_t* full, uint64_t* empty,
                            float4* meta, volatile Ctrl* ctrl, float4* pbuf, uint8_t* fillpar, int c0, int pw) {
    const KParams& p = cp.k;
    const int lane = threadIdx.x & 31;
    const int S = p.stages;
    const int per = S / kCsProd;   // stages this warp fills
    const int q = p.q;
    const int64_t total = p.rounds * (int64_t)q;
    const int64_t mine = total > pw ? (total - pw + kCsProd - 1) / kCsProd : 0;   // rows of this warp
    constexpr uint32_t eb = ELT == ELT_F32 ? 4u : (ELT == ELT_BF16 ? 2u : 1u);
    const uint8_t* Ac = p.A + (size_t)c0 * 4u * eb;
    const int nl = max(0, min(p.n4 - c0, cp.chunk));
    const uint32_t bytes = cs_copy_bytes<ELT>(nl);
    const uint64_t pol = policy_evict_first();
    int* status = &p.info->status;
    // rows issued at once: small chunks are bound by the copies' count (issue them together),
    // large ones by bandwidth (issue them in order, so that the first rows land first)
    const int lanes = bytes > 4096u ? 1 : (per < 32 ? per : 32);
    bool stop = false;
    for (int64_t base = 0; base < mine && !stop; base += 32) {
        const int64_t il = base + lane;
        if (il < mine) {
            const int64_t tl = il * kCsProd + pw;                    // sequence index
            const uint32_t own = (uint32_t)(tl % q);                 // worker j
            const uint64_t tt = (uint64_t)p.round0 + (uint64_t)(tl / q);
            uint32_t row = draw_row(p, p.same_stream ? 0u : own, tt);
            if (row >= p.m) {   // a row block of zero weight: nothing to draw
                set_status(status, RK_EINVAL);
                row = 0;
            }
            const float sc = (ELT == ELT_FP8) ? __ldg(p.row_scale + row) : 1.f;
            float wi = p.row_weight ? __ldg(p.row_weight + row) : 1.f;
            if (p.worker_weight) wi *= __ldg(p.worker_weight + own);
            pbuf[lane] = make_float4(__uint_as_float(row), __ldg(p.b + row), __ldg(p.inv + row) * wi, sc);
        }
        __syncwarp();
        // ... and issue them
        const int64_t rem_ = mine - base;
        const int cnt = rem_ < 32 ? (int)rem_ : 32;
        if (lanes == 1) {
            // in order, from lane 0, waiting for each stage in turn
            if (lane == 0) {
                for (int k = 0; k < cnt; ++k) {
                    const int64_t il = base + k;
                    const int64_t tt = il * kCsProd + pw;
                    const int st = pw + kCsProd * (int)(il % per);
                    const uint32_t ps = (uint32_t)((il / per) & 1);
                    if (tt >= ctrl->stop_t) { stop = true; break; }
                    if (tt >= S && !mbar_try_wait(&empty[st], ps ^ 1u)) {
                        // the previous copy into this stage (the last pass's) was consumed
                        const uint64_t t0 = globaltimer_ns();
                        while (!mbar_try_wait(&empty[st], ps ^ 1u)) {
                            if (tt >= ctrl->stop_t) { stop = true; break; }
                            if (globaltimer_ns() - t0 > p.timeout_ns) {
                                set_status(status, RK_ETIMEOUT);
                                stop = true;
                                break;
                            }
                        }
                        if (stop) break;
                    }
                    const float4 e = pbuf[k];
                    meta[st] = make_float4(e.y, e.z, e.w, 0.f);
                    if (bytes) {
                        mbar_arrive_expect_tx(&full[st], bytes);
                        bulk_g2s(stages + (size_t)st * p.stage_stride,
                                 Ac + (size_t)__float_as_uint(e.x) * (size_t)p.lda_bytes, bytes, &full[st], pol);
                    } else {
                        mbar_arrive(&full[st]);
                    }
                    fillpar[st] = (uint8_t)ps;
                }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            __syncwarp();
            continue;
        }
        // up to `lanes` <= `per` rows at once (distinct stages, each stage's empty barrier
        // at most one phase behind): every lane tests its own stage without blocking and
        // issues its copy when the stage is free; when none is free, the lane of the
        // oldest pending row (whose stage is released first) blocks on it alone
        for (int k0 = 0; k0 < cnt && !stop; k0 += lanes) {
            const int k = k0 + lane;
            const int64_t il = base + k;
            const int64_t tt = il * kCsProd + pw;
            const int st = pw + kCsProd * (int)(il % per);
            const uint32_t ps = (uint32_t)((il / per) & 1);
            bool pending = lane < lanes && k < cnt;
            while (__any_sync(0xffffffffu, pending)) {
                if (pending && tt >= ctrl->stop_t) {   // past what the consumers take
                    pending = false;
                    stop = true;
                }
                const bool ready = pending && (tt < S || cs_test_wait(&empty[st], ps ^ 1u));
                if (ready) {
                    const float4 e = pbuf[k];
                    meta[st] = make_float4(e.y, e.z, e.w, 0.f);
                    if (bytes) {
                        mbar_arrive_expect_tx(&full[st], bytes);
                        bulk_g2s(stages + (size_t)st * p.stage_stride,
                                 Ac + (size_t)__float_as_uint(e.x) * (size_t)p.lda_bytes, bytes, &full[st], pol);
                    } else {
                        mbar_arrive(&full[st]);
                    }
                    fillpar[st] = (uint8_t)ps;
                    pending = false;
                }
                const unsigned waiting = __ballot_sync(0xffffffffu, pending);
                if (waiting && !__any_sync(0xffffffffu, ready)) {
                    if (lane == __ffs(waiting) - 1) {
                        // the previous copy into this stage (the last pass's) was consumed
                        const uint64_t t0 = globaltimer_ns();
                        while (!mbar_try_wait(&empty[st], ps ^ 1u)) {
                            if (tt >= ctrl->stop_t) break;
                            if (globaltimer_ns() - t0 > p.timeout_ns) {
                                set_status(status, RK_ETIMEOUT);
                                stop = true;
                                break;
                            }
                        }
                    }
                    if (__any_sync(0xffffffffu, stop)) pending = false;   // a wait that ran out
                }
            }
            stop = __any_sync(0xffffffffu, stop);
        }
        __syncwarp();
    }
    // every copy this warp issued must land before the CTA exits: the last fill of
    // each of its stages
    __syncwarp();
    for (int i = lane; i < per; i += 32) {
        const int st = pw + kCsProd * i;
        if (fillpar[st] != 0xFFu) wait_parity(&full[st], fillpar[st], drain_limit_ns(p.timeout_ns), status);
    }
    __syncwarp();
}

// wait_parity with a short back-off between polls (the waits of this kernel are for
// rows a round ahead of the copies; tight polling only steals issue slots)
__device__ __forceinline__ bool cs_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns, int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        __nanosleep(64);
        if (globaltimer_ns() - t0 > timeout_ns) {
            set_status(status, RK_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// The partial dots of R (<= 8) staged rows against this CTA's chunk of x, the lanes of
// the warp taking consecutive slices (lane + 32 i): each lane's sums over its slices,
// acc[rr] for row rr.  Slices past the chunk read nothing; the row's last slice is
// masked past column n (its elements there are the row's padding).
template <int ELT, int R>
__device__ __forceinline__ void cs_dot_rows(const uint8_t* stages, const uint32_t* off, const float4* xs, int nl,
                                            bool has_tail, int rem, float* acc) {
    const int lane = threadIdx.x & 31;
    const int L = (nl + 31) >> 5;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) acc[rr] = 0.f;
    for (int i = 0; i + 1 < L; ++i) {
        const int idx = lane + 32 * i;
        const float4 xk = xs[idx];
        float4 a[R];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) a[rr] = load4<ELT>(stages + off[rr], idx);
#pragma unroll
        for (int rr = 0; rr < R; ++rr)
            acc[rr] = fmaf(a[rr].w, xk.w, fmaf(a[rr].z, xk.z, fmaf(a[rr].y, xk.y, fmaf(a[rr].x, xk.x, acc[rr]))));
    }
    const int idx = lane + 32 * (L - 1);
    if (L > 0 && idx < nl) {
        const float4 xk = xs[idx];
        const bool tail = has_tail && idx == nl - 1;
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
            float4 a = load4<ELT>(stages + off[rr], idx);
            if (tail) a = zero_beyond(a, rem);
            acc[rr] = fmaf(a.w, xk.w, fmaf(a.z, xk.z, fmaf(a.y, xk.y, fmaf(a.x, xk.x, acc[rr]))));
        }
    }
}

// Sums over the warp of eight per-lane values at once (a transposed butterfly: at
// each of the first three steps a lane keeps half of its values and sends the other
// half to its partner, 4 + 2 + 1 shuffles, then two plain steps).  Returns, in every
// lane l, the warp's total of value 4 b4 + 2 b3 + b2 (bk = bit k of l).  The order of
// the additions is fixed, so the result is the same on every run.
__device__ __forceinline__ float cs_reduce8(const float* acc) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = b4 ? acc[k] : acc[k + 4];
        const float keep = b4 ? acc[k + 4] : acc[k];
        h[k] = keep + __shfl_xor_sync(FULL, send, 16);
    }
    float t[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b3 ? h[k] : h[k + 2];
        const float keep = b3 ? h[k + 2] : h[k];
        t[k] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    float u;
    {
        const float send = b2 ? t[0] : t[1];
        const float keep = b2 ? t[1] : t[0];
        u = keep + __shfl_xor_sync(FULL, send, 4);
    }
    u += __shfl_xor_sync(FULL, u, 2);
    u += __shfl_xor_sync(FULL, u, 1);
    return u;
}

template <int NT, int ELT>
__global__ void __launch_bounds__(NT + 32 * kCsProd, 1) rka_colsplit_kernel(const CSParams cp) {
    const KParams& p = cp.k;
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int NW = NT / 32;
    constexpr int RB = kCsMaxQ / NW;   // rows a warp in the dot pass, at most
    static_assert(RB <= 8, "the dot pass reduces at most eight rows a warp");
    const int S = p.stages;
    const int q = p.q;
    const bool warp_rows = cp.warp_rows != 0;
    const uint32_t stride = p.stage_stride;
    uint8_t* stages = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * stride);
    uint64_t* empty = full + S;
    float4* meta = reinterpret_cast<float4*>(empty + S);
    float4* xs = meta + S;                                        // [XP]
    float4* dpart = xs + (cp.chunk + 31) / 32 * 32;               // [NW][chunk] with warp rows
    float4* grp = dpart + (warp_rows ? (size_t)NW * cp.chunk : 0);   // [NT / 16][16]
    float2* rowc = reinterpret_cast<float2*>(grp + NT);           // [kCsMaxQ]
    double* chk = reinterpret_cast<double*>(rowc + kCsMaxQ);      // [96]
    float4* pbuf = reinterpret_cast<float4*>(chk + 96);           // [kCsProd][32] the producers' draws
    volatile Ctrl* ctrl = reinterpret_cast<volatile Ctrl*>(pbuf + 32 * kCsProd);
    uint8_t* fillpar = reinterpret_cast<uint8_t*>(pbuf + 32 * kCsProd) + 16;   // [S] parity of each stage's last fill

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int G = (int)gridDim.x;
    const int g = (int)blockIdx.x;
    const int c0 = g * cp.chunk;                          // first slice of x this CTA owns
    const int nl = max(0, min(p.n4 - c0, cp.chunk));      // slices it owns
    const int64_t total = p.rounds * (int64_t)q;
    int* status = &p.info->status;

    {
        uint4* z = reinterpret_cast<uint4*>(stages);
        const size_t nz = (size_t)S * stride / 16;
        for (size_t i = tid; i < nz; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);    // the issuing lane's arrive with the copy's byte count
            mbar_init(&empty[i], warp_rows ? 1 : NW);   // the readers of a stage's row
            fillpar[i] = 0xFFu;        // never filled
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
    if (p.sampling == RK_SAMPLE_CYCLIC && p.setup->range_rows != 0) {
        if (tid == 0) set_status(status, RK_EINVAL);
        return;
    }
    if (warp >= NW) {
        const int pw = warp - NW;
        cs_producer<ELT>(cp, stages, full, empty, meta, ctrl, pbuf + 32 * pw, fillpar, c0, pw);
        return;
    }

    // ---------------- consumers ----------------
    const int rem = p.n & 3;
    const bool has_tail = rem != 0 && nl > 0 && c0 + nl == p.n4;   // the row's last slice is this CTA's
    // this CTA's chunk of x (the round's start point), zero past column n and past the chunk
    for (int s = tid; s < (nl + 31) / 32 * 32; s += NT) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s < nl) {
            const int j = (c0 + s) * 4;
            t.x = __ldg(p.x0 + j);
            if (j + 1 < p.n) t.y = __ldg(p.x0 + j + 1);
            if (j + 2 < p.n) t.z = __ldg(p.x0 + j + 2);
            if (j + 3 < p.n) t.w = __ldg(p.x0 + j + 3);
        }
        xs[s] = t;
    }
    named_bar_sync(1, NT);
    const float rq = 1.0f / (float)q;
    const int cnt = q > warp ? (q - warp + NW - 1) / NW : 0;   // rows j = warp, warp + NW, ... of this warp
    int64_t u = 0;                 // sequence index of the round's first row
    int s0 = 0;                    // its stage (u mod S) ...
    uint32_t ph0 = 0;              // ... and the parity of its pass over the ring
    // stage and parity of the round's row j (j < q <= S: at most one wrap)
    auto stage_of = [&](int j, uint32_t& par) {
        int st = s0 + j;
        par = ph0;
        if (st >= S) { st -= S; par ^= 1u; }
        return st;
    };
    unsigned long long nbar = 0;   // grid barriers passed
    bool ok = true;
    for (int64_t r = 0; r < p.rounds && ok; ++r) {
        const int rb = (int)(r & 1);
        // ---- 1. partial dots: each warp forms its rows whole over the chunk ----
        bool got = true;
        uint32_t off[RB];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) {
            off[rr] = 0;
            if (rr < cnt) {
                uint32_t par;
                const int st = stage_of(warp + NW * rr, par);
                got = cs_wait(&full[st], par, p.timeout_ns, status) && got;
                off[rr] = (uint32_t)st * stride;
            }
        }
        float acc[8];
        switch (cnt) {
            case 8: cs_dot_rows<ELT, (RB >= 8 ? 8 : RB)>(stages, off, xs, nl, has_tail, rem, acc); break;
            case 7: cs_dot_rows<ELT, (RB >= 7 ? 7 : RB)>(stages, off, xs, nl, has_tail, rem, acc); break;
            case 6: cs_dot_rows<ELT, (RB >= 6 ? 6 : RB)>(stages, off, xs, nl, has_tail, rem, acc); break;
            case 5: cs_dot_rows<ELT, (RB >= 5 ? 5 : RB)>(stages, off, xs, nl, has_tail, rem, acc); break;
            case 4: cs_dot_rows<ELT, (RB >= 4 ? 4 : RB)>(stages, off, xs, nl, has_tail, rem, acc); break;
            case 3: cs_dot_rows<ELT, (RB >= 3 ? 3 : RB)>(stages, off, xs, nl, has_tail, rem, acc); break;
            case 2: cs_dot_rows<ELT, 2>(stages, off, xs, nl, has_tail, rem, acc); break;
            case 1: cs_dot_rows<ELT, 1>(stages, off, xs, nl, has_tail, rem, acc); break;
            default:
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) acc[rr] = 0.f;
        }
        {
            const float sum = cs_reduce8(acc);
            const int rr = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
            if ((lane & 3) == 0 && rr < cnt) cp.part[((size_t)rb * G + g) * kCsMaxQ + warp + NW * rr] = sum;
        }
        // ---- 2. one grid barrier (the CTA barrier orders every warp's partials before it) ----
        if (!bar_and(1, NT, got)) { ok = false; break; }
        if (tid == 0)
            ctrl->flag = grid_sync(&p.info->bar_arrivals, nbar, (unsigned)G, status, p.timeout_ns) ? 1 : 0;
        ++nbar;
        named_bar_sync(1, NT);
        if (!ctrl->flag) { ok = false; break; }
        // ---- 3. <A_j, x> = sum_g p_j^g in a fixed order, the coefficients ----
        // thread (h, f) sums float4 f (workers 4f .. 4f+3) of the CTAs g = h, h + H, ...
        // in ascending g, all its loads in flight at once; then each worker's total is
        // the sum over h in ascending order: the same order in every CTA
        {
            constexpr int H = NT / 16;
            constexpr int B = 16;   // loads in flight a thread
            const int f = tid & 15, h = tid >> 4;
            const float4* pr4 = reinterpret_cast<const float4*>(cp.part + (size_t)rb * G * kCsMaxQ);
            float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * f < q) {
                for (int g0 = h; g0 < G; g0 += H * B) {
                    float4 w[B];
#pragma unroll
                    for (int e = 0; e < B; ++e) {
                        const int gg = g0 + e * H;
                        w[e] = gg < G ? __ldcg(pr4 + (size_t)gg * (kCsMaxQ / 4) + f) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int e = 0; e < B; ++e) {
                        t4.x += w[e].x; t4.y += w[e].y; t4.z += w[e].z; t4.w += w[e].w;
                    }
                }
            }
            grp[h * 16 + f] = t4;
        }
        named_bar_sync(1, NT);
        for (int j = tid; j < q; j += NT) {
            const float* gj = reinterpret_cast<const float*>(grp) + j;   // component j % 4 of float4 j / 4
            float dot = 0.f;
            for (int h = 0; h < NT / 16; ++h) dot += gj[h * 64];
            uint32_t par;
            const int st = stage_of(j, par);
            const float4 mb = meta[st];   // b_j, w_j / ||A_j||^2, row scale s_j
            // A_j = s_j q_j: <A_j, x> = s_j <q_j, x>, and the update takes (c_j s_j) q_j
            rowc[j] = make_float2(p.omega * (mb.x - mb.z * dot) * mb.y * mb.z, __uint_as_float((uint32_t)st * stride));
        }
        named_bar_sync(1, NT);
        // ---- 4. d = sum_j c_j A_j[chunk], x += d / q ----
        if (warp_rows) {
            // warp w sums its own rows j = w, w + NW, ... (ascending) over the chunk's
            // slices lane + 32 i into dpart[w]; the NW sums are then added in ascending w
            float2 rc[8];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) rc[rr] = rr < cnt ? rowc[warp + NW * rr] : make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < kCsWarpRowsL; ++i) {
                const int sl = lane + 32 * i;
                if (sl < nl) {
                    float4 dd = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        if (rr < cnt) {
                            const float4 av = load4<ELT>(stages + __float_as_uint(rc[rr].y), sl);
                            const float2 c2 = make_float2(rc[rr].x, rc[rr].x);
                            const float2 lo = __ffma2_rn(c2, make_float2(av.x, av.y), make_float2(dd.x, dd.y));
                            const float2 hi = __ffma2_rn(c2, make_float2(av.z, av.w), make_float2(dd.z, dd.w));
                            dd = make_float4(lo.x, lo.y, hi.x, hi.y);
                        }
                    }
                    // the row's padding past column n never reaches x
                    if (has_tail && sl == nl - 1) dd = zero_beyond(dd, rem);
                    dpart[(size_t)warp * cp.chunk + sl] = dd;
                }
            }
            __syncwarp();
            // this warp alone read its rows' stages: release them
            if (lane < cnt) {
                uint32_t par;
                mbar_arrive(&empty[stage_of(warp + NW * lane, par)]);
            }
            named_bar_sync(1, NT);
            for (int sl = tid; sl < nl; sl += NT) {
                float4 dd = dpart[sl];
#pragma unroll
                for (int w = 1; w < NW; ++w) {
                    const float4 t = dpart[(size_t)w * cp.chunk + sl];
                    dd.x += t.x; dd.y += t.y; dd.z += t.z; dd.w += t.w;
                }
                const float4 v = xs[sl];
                xs[sl] = make_float4(fmaf(dd.x, rq, v.x), fmaf(dd.y, rq, v.y), fmaf(dd.z, rq, v.z), fmaf(dd.w, rq, v.w));
            }
        } else {
            // slices sl = tid + NT i of every thread, each summed over all rows in ascending j,
            // UJ rows a step with their coefficients and slices loaded together
            constexpr int UJ = 8;
            if (nl <= kCsSlicesAThread * NT) {
                // rows outer: after each step every warp has read the step's rows and
                // releases their stages, so that the next round's copies can land while the
                // update goes on (rings of one round, the widest chunks)
                float4 dd[kCsSlicesAThread];
#pragma unroll
                for (int i = 0; i < kCsSlicesAThread; ++i) dd[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int j0 = 0; j0 < q; j0 += UJ) {
                    const int jc = min(UJ, q - j0);   // rows of this step
                    float2 rcj[UJ];
#pragma unroll
                    for (int e = 0; e < UJ; ++e) rcj[e] = e < jc ? rowc[j0 + e] : make_float2(0.f, 0.f);
#pragma unroll
                    for (int i = 0; i < kCsSlicesAThread; ++i) {
                        const int sl = tid + NT * i;
                        if (sl < nl) {
                            float4 av[UJ];
#pragma unroll
                            for (int e = 0; e < UJ; ++e)
                                av[e] = e < jc ? load4<ELT>(stages + __float_as_uint(rcj[e].y), sl)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                            for (int e = 0; e < UJ; ++e) {
                                if (e < jc) {
                                    const float2 c2 = make_float2(rcj[e].x, rcj[e].x);
                                    const float2 lo = __ffma2_rn(c2, make_float2(av[e].x, av[e].y),
                                                                 make_float2(dd[i].x, dd[i].y));
                                    const float2 hi = __ffma2_rn(c2, make_float2(av[e].z, av[e].w),
                                                                 make_float2(dd[i].z, dd[i].w));
                                    dd[i] = make_float4(lo.x, lo.y, hi.x, hi.y);
                                }
                            }
                        }
                    }
                    __syncwarp();
                    if (lane < jc) {
                        uint32_t par;
                        mbar_arrive(&empty[stage_of(j0 + lane, par)]);
                    }
                }
#pragma unroll
                for (int i = 0; i < kCsSlicesAThread; ++i) {
                    const int sl = tid + NT * i;
                    if (sl < nl) {
                        if (has_tail && sl == nl - 1) dd[i] = zero_beyond(dd[i], rem);
                        const float4 v = xs[sl];
                        xs[sl] = make_float4(fmaf(dd[i].x, rq, v.x), fmaf(dd[i].y, rq, v.y), fmaf(dd[i].z, rq, v.z),
                                             fmaf(dd[i].w, rq, v.w));
                    }
                }
            } else {
                for (int sl = tid; sl < nl; sl += NT) {
                    float4 dd = make_float4(0.f, 0.f, 0.f, 0.f);
                    int j = 0;
                    for (; j + UJ <= q; j += UJ) {
                        float2 rcj[UJ];
                        float4 av[UJ];
#pragma unroll
                        for (int e = 0; e < UJ; ++e) rcj[e] = rowc[j + e];
#pragma unroll
                        for (int e = 0; e < UJ; ++e) av[e] = load4<ELT>(stages + __float_as_uint(rcj[e].y), sl);
#pragma unroll
                        for (int e = 0; e < UJ; ++e) {
                            const float2 c2 = make_float2(rcj[e].x, rcj[e].x);
                            const float2 lo = __ffma2_rn(c2, make_float2(av[e].x, av[e].y), make_float2(dd.x, dd.y));
                            const float2 hi = __ffma2_rn(c2, make_float2(av[e].z, av[e].w), make_float2(dd.z, dd.w));
                            dd = make_float4(lo.x, lo.y, hi.x, hi.y);
                        }
                    }
                    for (; j < q; ++j) {
                        const float2 rcj = rowc[j];
                        const float4 av = load4<ELT>(stages + __float_as_uint(rcj.y), sl);
                        const float2 c2 = make_float2(rcj.x, rcj.x);
                        const float2 lo = __ffma2_rn(c2, make_float2(av.x, av.y), make_float2(dd.x, dd.y));
                        const float2 hi = __ffma2_rn(c2, make_float2(av.z, av.w), make_float2(dd.z, dd.w));
                        dd = make_float4(lo.x, lo.y, hi.x, hi.y);
                    }
                    if (has_tail && sl == nl - 1) dd = zero_beyond(dd, rem);
                    const float4 v = xs[sl];
                    xs[sl] = make_float4(fmaf(dd.x, rq, v.x), fmaf(dd.y, rq, v.y), fmaf(dd.z, rq, v.z), fmaf(dd.w, rq, v.w));
                }
                __syncwarp();
                // every warp read every row: this warp's release of the round's stages
                for (int j = lane; j < q; j += 32) {
                    uint32_t par;
                    mbar_arrive(&empty[stage_of(j, par)]);
                }
            }
        }
        u += q;
        s0 += q;
        if (s0 >= S) { s0 -= S; ph0 ^= 1u; }
        named_bar_sync(1, NT);   // x complete for the next round's dots
        // ---- 5. convergence / divergence check (a second grid barrier) ----
        const int64_t done = r + 1;
        const bool last = (done == p.rounds);
        const bool check = p.check_every > 0 && (done % p.check_every == 0 || last);
        if (check) {
            ChkAcc ca{0.f, 0.f, 0.f};
            for (int s = tid; s < nl; s += NT) {
                const int j = (c0 + s) * 4;
                const float4 v = xs[s];
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (j + e < p.n) {
                        ca.xx = fmaf(vv[e], vv[e], ca.xx);
                        if (p.criterion == 1) {
                            const float xr = __ldg(p.x_ref + j + e);
                            const float dd = vv[e] - xr;
                            ca.e2 = fmaf(dd, dd, ca.e2);
                            ca.r2 = fmaf(xr, xr, ca.r2);
                        }
                    }
                }
            }
            check_warp_partials<NT>(ca, chk);
            named_bar_sync(1, NT);
            if (tid == 0) {
                check_cta_partial<NT>(p, chk);
                ctrl->flag = grid_sync(&p.info->bar_arrivals, nbar, (unsigned)G, status, p.timeout_ns) ? 1 : 0;
            }
            ++nbar;
            named_bar_sync(1, NT);
            if (!ctrl->flag) { ok = false; break; }
            combine_check<NT>(p, chk);
            const float* sh = reinterpret_cast<const float*>(chk);
            const float XX = sh[0], E2 = sh[1], R2 = sh[2];
            named_bar_sync(1, NT);
            float mf = -1.f;
            if (p.criterion == 1) mf = (R2 > 0.f) ? sqrtf(E2 / R2) : sqrtf(E2);
            const double metric = (double)mf;
            const bool diverged = !isfinite(XX) || (p.criterion == 1 && !isfinite(mf));
            if (g == 0 && tid == 0) {
                p.info->rounds_done = done;
                p.info->last_metric = metric;
            }
            if (diverged) {
                if (tid == 0) set_status(status, RK_EDIVERGED);
                ok = false;
            } else if (p.criterion == 1 && p.tol > 0.0 && metric < p.tol) {
                break;   // converged: the same decision in every CTA
            }
        } else if (g == 0 && tid == 0) {
            p.info->rounds_done = done;
        }
    }
    // stop the producer at what was consumed, and write this CTA's chunk of x
    if (tid == 0) ctrl->stop_t = u;
    named_bar_sync(1, NT);
    for (int s = tid; s < nl; s += NT) {
        const int j = (c0 + s) * 4;
        const float4 v = xs[s];
        p.x[j] = v.x;
        if (j + 1 < p.n) p.x[j + 1] = v.y;
        if (j + 2 < p.n) p.x[j + 2] = v.z;
        if (j + 3 < p.n) p.x[j + 3] = v.w;
    }
}

typedef void (*CsKernelFn)(const CSParams);

struct CsVariant {
    int elt;
    CsKernelFn fn;
};

// 256 consumer threads: eight rows a warp in the dot pass at 64 workers a round, and
// the grid reduction of each round wants many loads in flight
constexpr int kCsNT = 256;
#define CS_(ELT) CsVariant{ELT, rka_colsplit_kernel<kCsNT, ELT>}
static const CsVariant kCsTab[] = {CS_(ELT_F32), CS_(ELT_BF16), CS_(ELT_FP8)};
#undef CS_

int launch_colsplit_solve(const SolveArgs& a, const KParams& base, cudaStream_t st, int smem_max, int sms) {
    const Plan* pl = a.plan;
    if (a.q < 1 || a.q > kCsMaxQ) return RK_EINVAL;
    const int n4 = base.n4;
    const int chunk = ((n4 + sms - 1) / sms + 3) / 4 * 4;
    const int grid = (n4 + chunk - 1) / chunk;
    const int nt = kCsNT;
    const int elt = pl->dt == RK_F32 ? ELT_F32 : (pl->dt == RK_BF16 ? ELT_BF16 : ELT_FP8);
    const CsVariant* var = nullptr;
    for (const CsVariant& v : kCsTab)
        if (v.elt == elt) var = &v;
    if (!var) return RK_EINVAL;
    // the update: a warp's own rows over chunks of at most 128 slices (no thread idle in
    // a warp, stages released by their one reader), a thread's slices over all rows beyond
    const bool warp_rows = chunk <= kCsWarpRowsL * 32;
    const uint32_t eb = pl->dt == RK_F32 ? 4u : (pl->dt == RK_BF16 ? 2u : 1u);
    // a stage holds one chunk (the kernel reads no slice past the CTA's own)
    const uint32_t stride = ((uint32_t)chunk * 4u * eb + 127u) & ~127u;
    // every stage of a round stays taken until its update: at least q stages; up to
    // twice that lets the producer fetch the next round during the exchange
    int S = 0;
    while (S < 2 * a.q + kCsSpare && S < 252 &&
           (size_t)(S + 1) * stride + cs_ctrl_bytes(S + 1, nt, chunk, warp_rows) <= (size_t)smem_max)
        ++S;
    S -= S % kCsProd;   // each producer warp serves its own stages
    if (S < a.q) return RK_EINVAL;   // the round's rows do not fit the shared memory
    // partial dots (2 x grid x kCsMaxQ floats) and the per-CTA check partials (grid
    // float4) in the V block of the solve workspace: (v_rows + 1) x ldv floats
    const size_t part_floats = (size_t)2 * grid * kCsMaxQ;
    const size_t have = (size_t)(v_rows_for(a.q, a.alpha) + 1) * (size_t)a.ldv;
    if (part_floats + (size_t)grid * 4 + 4 > have) return RK_EINVAL;
    CSParams cp;
    cp.k = base;
    cp.k.stages = S;
    cp.k.stage_stride = stride;
    cp.k.row_bytes = 0;   // per-CTA copy sizes are computed in the kernel
    cp.k.chkpart = a.V + ((part_floats + 3) & ~(size_t)3);
    cp.chunk = chunk;
    cp.warp_rows = warp_rows ? 1 : 0;
    cp.part = a.V;
    const size_t smem = (size_t)S * stride + cs_ctrl_bytes(S, nt, chunk, warp_rows);
    if (cudaFuncSetAttribute(var->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RK_ECUDA;
    void* args[] = {(void*)&cp};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)var->fn, dim3((unsigned)grid),
                                                dim3((unsigned)(nt + 32 * kCsProd)), args, smem, st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        return RK_ENOTCORESIDENT;
    }
    if (e != cudaSuccess) return RK_ECUDA;
    count_launch();
    return RK_OK;
}

}  // namespace rk
