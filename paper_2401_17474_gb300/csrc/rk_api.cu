// rk_api.cu -- the extern "C" entry points declared in include/rkab.h:
// argument checks, workspace layouts, plan lifecycle and status reads.  All
// device work is in rk_setup.cu, rk_solve.cu and rk_residual.cu.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <new>

#include "rk_internal.h"

namespace rk {

static std::atomic<uint64_t> g_launches{0};

void count_launch(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static size_t elem_bytes(rk_dtype dt) {
    switch (dt) {
        case RK_F32: return 4;
        case RK_BF16: return 2;
        case RK_FP8E4M3: return 1;
    }
    return 0;
}

size_t setup_ws_bytes(int64_t m) {
    const size_t M = (size_t)m;
    return align256(sizeof(SetupInfo))     // info
           + align256(M * 8) * 3           // K, P, thr64
           + align256(M * 4) * 2           // alias, inv
           + align256(M * 16)              // R
           + align256(M * 4)               // e
           + align256(M * 4)               // row_pos
           + align256(M * 16) * 3          // row_Dex, light_Dinc, heavy_Einc
           + align256(M * 4)               // heavy_idx
           + align256(scan_tiles_bytes(m)) // scan tile sums
           + align256(scan_item_bytes());  // scan total
}

SetupWs setup_ws_carve(void* base, int64_t m) {
    const size_t M = (size_t)m;
    uint8_t* p = static_cast<uint8_t*>(base);
    SetupWs w;
    auto take = [&](size_t bytes) {
        uint8_t* q = p;
        p += align256(bytes);
        return q;
    };
    w.info = reinterpret_cast<SetupInfo*>(take(sizeof(SetupInfo)));
    w.K = reinterpret_cast<uint64_t*>(take(M * 8));
    w.P = reinterpret_cast<uint64_t*>(take(M * 8));
    w.thr64 = reinterpret_cast<uint64_t*>(take(M * 8));
    w.alias = reinterpret_cast<uint32_t*>(take(M * 4));
    w.inv = reinterpret_cast<float*>(take(M * 4));
    w.R = reinterpret_cast<u128*>(take(M * 16));
    w.e = reinterpret_cast<int*>(take(M * 4));
    w.row_pos = reinterpret_cast<uint32_t*>(take(M * 4));
    w.row_Dex = reinterpret_cast<u128*>(take(M * 16));
    w.light_Dinc = reinterpret_cast<u128*>(take(M * 16));
    w.heavy_Einc = reinterpret_cast<u128*>(take(M * 16));
    w.heavy_idx = reinterpret_cast<uint32_t*>(take(M * 4));
    w.tiles = take(scan_tiles_bytes(m));
    w.tile_total = take(scan_item_bytes());
    return w;
}

// Row selection: a known mode; per-worker modes need the workers' own streams.
bool sampling_ok(const rk_opts& o) {
    if (o.sampling == RK_SAMPLE_FULL) return true;
    return (o.sampling == RK_SAMPLE_BLOCKS || o.sampling == RK_SAMPLE_CYCLIC) && !o.same_stream;
}

// Options every solve entry point accepts (rkab_solve, rkab_solve_noalloc, and the
// solves inside rkab_solve_residual and rkab_adjoint).
bool solve_opts_valid(const rk_opts& o, int q) {
    return omega_ok(o.omega, q) && sampling_ok(o) && o.check_every >= 0 && o.round0 >= 0 &&
           o.timeout_s > 0.0 && !(o.criterion == 1 && !o.x_ref) && o.criterion >= 0 &&
           o.criterion <= 1 &&
           (o.lookahead == 0 || o.lookahead == 1 || o.lookahead == 2 || o.lookahead == 4 ||
            o.lookahead == 6) &&
           o.cluster_size >= 0 && o.cluster_size <= 16 && (o.cluster_size & (o.cluster_size - 1)) == 0;
}

}  // namespace rk

using namespace rk;

extern "C" {

void rk_opts_default(rk_opts* o) {
    if (!o) return;
    o->omega = 1.0f;
    o->check_every = 1;
    o->tol = 0.0;
    o->criterion = 0;
    o->x_ref = nullptr;
    o->round0 = 0;
    o->stream_id = 0;
    o->same_stream = 0;
    o->cluster_size = 0;
    o->timeout_s = 10.0;
    o->lookahead = 0;
    o->sampling = RK_SAMPLE_FULL;
    o->row_weight = nullptr;
    o->worker_weight = nullptr;
}

const char* rk_strerror(int code) {
    switch (code) {
        case RK_OK: return "ok";
        case RK_EINVAL: return "invalid argument";
        case RK_EALIGN: return "address or leading dimension not 16-byte aligned";
        case RK_ENOTCORESIDENT: return "persistent grid does not fit co-resident on the device";
        case RK_ETIMEOUT: return "device-side wait exceeded its time limit";
        case RK_EDIVERGED: return "iterate became non-finite";
        case RK_ECUDA: return "CUDA runtime error";
        case RK_EWORKSPACE: return "workspace too small";
        case RK_ESETUP: return "plan setup failed on the device (non-finite or all-zero matrix, or a "
                               "row with ||A_i||^2 outside the float32 range)";
        case RK_ETOOLARGE: return "q x n exceeds the fixed scratch of the allocation-free solve";
        default: return "unknown error";
    }
}

uint64_t rk_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

size_t rk_setup_workspace_bytes(int64_t m, int64_t n) {
    (void)n;
    if (m < 1) return 0;
    return setup_ws_bytes(m);
}

int rk_setup(const void* A, rk_dtype dt, const float* row_scale, int64_t m, int64_t n,
             int64_t lda, void* workspace, size_t ws_bytes, void* stream, rk_plan** out) {
    if (!out) return RK_EINVAL;
    *out = nullptr;
    if (!A || !workspace || m < 1 || n < 1 || lda < n) return RK_EINVAL;
    if (m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 26)) return RK_EINVAL;
    const size_t eb = elem_bytes(dt);
    if (eb == 0) return RK_EINVAL;
    if (dt == RK_FP8E4M3 && !row_scale) return RK_EINVAL;
    if (!aligned16(A) || ((size_t)lda * eb) % 16 != 0) return RK_EALIGN;
    if (((uintptr_t)workspace & 255u) != 0) return RK_EALIGN;
    if (ws_bytes < setup_ws_bytes(m)) return RK_EWORKSPACE;
    rk_plan* pl = new (std::nothrow) rk_plan;
    if (!pl) return RK_EINVAL;
    pl->p.A = A;
    pl->p.dt = dt;
    pl->p.row_scale = row_scale;
    pl->p.m = m;
    pl->p.n = n;
    pl->p.lda = lda;
    pl->p.ws = setup_ws_carve(workspace, m);
    const int rc = launch_setup(A, dt, row_scale, m, n, lda, pl->p.ws,
                                static_cast<cudaStream_t>(stream));
    if (rc != RK_OK) {
        delete pl;
        return rc;
    }
    *out = pl;
    return RK_OK;
}

int rk_plan_status(const rk_plan* plan, void* stream, uint64_t* T_out, int32_t* L_out) {
    if (!plan) return RK_EINVAL;
    SetupInfo info;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&info, plan->p.ws.info, sizeof(info), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RK_ECUDA;
    if (info.status != 0 || info.H == kNoRows || info.T == 0) return RK_ESETUP;
    if (T_out) *T_out = info.T;
    if (L_out) *L_out = info.L;
    return RK_OK;
}

int rk_plan_tables(const rk_plan* plan, const uint64_t** K, const uint64_t** P,
                   const uint64_t** thr64, const uint32_t** alias, const float** inv) {
    if (!plan) return RK_EINVAL;
    if (K) *K = plan->p.ws.K;
    if (P) *P = plan->p.ws.P;
    if (thr64) *thr64 = plan->p.ws.thr64;
    if (alias) *alias = plan->p.ws.alias;
    if (inv) *inv = plan->p.ws.inv;
    return RK_OK;
}

void rk_plan_destroy(rk_plan* plan) { delete plan; }

int rk_sample_indices(const rk_plan* plan, uint64_t seed, uint32_t worker, uint32_t stream_id,
                      uint64_t t0, int64_t count, uint32_t* out, void* stream) {
    if (!plan || count < 0 || (count > 0 && !out)) return RK_EINVAL;
    return launch_sample_indices(&plan->p, seed, worker, stream_id, t0, count, out,
                                 static_cast<cudaStream_t>(stream));
}

int rk_sample_indices_ex(const rk_plan* plan, uint64_t seed, uint32_t worker, uint32_t q,
                         uint32_t stream_id, int sampling, uint64_t t0, int64_t count,
                         uint32_t* out, void* stream) {
    if (!plan || count < 0 || (count > 0 && !out) || q < 1 || worker >= q ||
        (sampling != RK_SAMPLE_FULL && sampling != RK_SAMPLE_BLOCKS && sampling != RK_SAMPLE_CYCLIC))
        return RK_EINVAL;
    return launch_sample_indices_ex(&plan->p, seed, worker, q, stream_id, sampling, t0, count, out,
                                    static_cast<cudaStream_t>(stream));
}

size_t rk_solve_workspace_bytes(const rk_plan* plan, int q) {
    if (!plan || q < 1) return 0;
    return solve_ws_bytes(&plan->p, q);
}

int rkab_solve(const rk_plan* plan, const float* b, const float* x0, float* x, int q,
               int64_t alpha, int64_t rounds, uint64_t seed, const rk_opts* opts,
               void* workspace, size_t ws_bytes, void* stream) {
    if (!plan || !b || !x0 || !x || !workspace || q < 1 || alpha < 1 || rounds < 0)
        return RK_EINVAL;
    rk_opts o;
    rk_opts_default(&o);
    if (opts) o = *opts;
    if (!solve_opts_valid(o, q)) return RK_EINVAL;
    if (((uintptr_t)workspace & 255u) != 0) return RK_EALIGN;
    if (ws_bytes < solve_ws_bytes(&plan->p, q)) return RK_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SolveInfo* info = static_cast<SolveInfo*>(workspace);
    if (cudaMemsetAsync(info, 0, sizeof(SolveInfo), st) != cudaSuccess) return RK_ECUDA;
    if (rounds == 0) {
        if (x != x0 &&
            cudaMemcpyAsync(x, x0, (size_t)plan->p.n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return RK_ECUDA;
        return RK_OK;
    }
    SolveArgs a;
    a.plan = &plan->p;
    a.b = b;
    a.x0 = x0;
    a.x = x;
    a.q = q;
    a.alpha = alpha;
    a.rounds = rounds;
    a.seed = seed;
    a.opts = o;
    a.info = info;
    const int64_t n4 = (plan->p.n + 3) / 4;
    a.ldv = n4 * 4;
    a.V = reinterpret_cast<float*>(static_cast<uint8_t*>(workspace) + align256(sizeof(SolveInfo)));
    return launch_solve(a, st);
}

int rka_solve(const rk_plan* plan, const float* b, const float* x0, float* x, int q,
              int64_t rounds, uint64_t seed, const rk_opts* opts, void* workspace,
              size_t ws_bytes, void* stream) {
    return rkab_solve(plan, b, x0, x, q, 1, rounds, seed, opts, workspace, ws_bytes, stream);
}

int rk_solve_status(const void* workspace, void* stream, int64_t* rounds_done,
                    double* last_metric) {
    if (!workspace) return RK_EINVAL;
    SolveInfo info;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&info, workspace, sizeof(info), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RK_ECUDA;
    if (rounds_done) *rounds_done = info.rounds_done;
    if (last_metric) *last_metric = info.last_metric;
    return info.status;
}

int rk_quantize(const float* A, int64_t m, int64_t n, int64_t lda, rk_dtype dt, void* out,
                int64_t ldo, float* row_scale, void* stream) {
    if (!A || !out || m < 1 || n < 1 || lda < n || ldo < n) return RK_EINVAL;
    if (dt != RK_BF16 && dt != RK_FP8E4M3) return RK_EINVAL;
    if (dt == RK_FP8E4M3 && !row_scale) return RK_EINVAL;
    if (!aligned16(out) || ((size_t)ldo * elem_bytes(dt)) % 16 != 0) return RK_EALIGN;
    return launch_quantize(A, m, n, lda, dt, out, ldo, row_scale, static_cast<cudaStream_t>(stream));
}

size_t rk_refine_workspace_bytes(const rk_plan* lowp, int q) {
    if (!lowp || q < 1) return 0;
    return refine_ws_bytes(&lowp->p, q);
}

int rkab_refine(const rk_plan* lowp, const float* A32, int64_t lda32, const float* b,
                const float* x0, float* x, int q, int64_t alpha, int64_t inner_rounds,
                int64_t max_outer, uint64_t seed, const rk_opts* opts, void* workspace,
                size_t ws_bytes, void* stream, int64_t* outer_done, double* last_metric) {
    if (!lowp || !A32 || !b || !x0 || !x || !workspace || q < 1 || alpha < 1 ||
        inner_rounds < 1 || max_outer < 0 || lda32 < lowp->p.n)
        return RK_EINVAL;
    if (!aligned16(A32) || (lda32 * 4) % 16 != 0 || ((uintptr_t)workspace & 255u) != 0)
        return RK_EALIGN;
    rk_opts o;
    rk_opts_default(&o);
    if (opts) o = *opts;
    if (!omega_ok(o.omega, q) || !(o.timeout_s > 0.0) ||
        (o.criterion == 1 && !o.x_ref) || o.criterion < 0 || o.criterion > 1 || !sampling_ok(o))
        return RK_EINVAL;
    if (ws_bytes < refine_ws_bytes(&lowp->p, q)) return RK_EWORKSPACE;
    return run_refine(&lowp->p, A32, lda32, b, x0, x, q, alpha, inner_rounds, max_outer, seed, o,
                      workspace, static_cast<cudaStream_t>(stream), outer_done, last_metric);
}

int rk_transpose(const float* A, int64_t m, int64_t n, int64_t lda, float* At, int64_t ldt,
                 void* stream) {
    if (!A || !At || m < 1 || n < 1 || lda < n || ldt < m) return RK_EINVAL;
    if (!aligned16(At) || (ldt * 4) % 16 != 0) return RK_EALIGN;
    return launch_transpose(A, m, n, lda, At, ldt, static_cast<cudaStream_t>(stream));
}

int rk_rank2(const float* r, const float* g, const float* y, const float* x, int64_t m, int64_t n,
             float* G, int64_t ldg, void* stream) {
    if (!r || !g || !y || !x || !G || m < 1 || n < 1 || ldg < n) return RK_EINVAL;
    if (!aligned16(G) || (ldg * 4) % 16 != 0) return RK_EALIGN;
    return launch_rank2(r, g, y, x, m, n, G, ldg, static_cast<cudaStream_t>(stream));
}

size_t rk_adjoint_workspace_bytes(const rk_plan* plan_A, const rk_plan* plan_At, int q_t, int q) {
    if (!plan_A || !plan_At || q < 1 || q_t < 1) return 0;
    return adjoint_ws_bytes(&plan_A->p, &plan_At->p, q_t, q);
}

int rkab_adjoint(const rk_plan* plan_A, const rk_plan* plan_At, const float* b, const float* x,
                 const float* gx, int q_t, int q, int64_t alpha_t, int64_t rounds_t, int64_t alpha,
                 int64_t rounds, uint64_t seed, const rk_opts* opts_t, const rk_opts* opts,
                 float* grad_b, float* g, float* grad_A, int64_t ldg, void* workspace,
                 size_t ws_bytes, void* stream) {
    if (!plan_A || !plan_At || !b || !x || !gx || !grad_b || !g || !grad_A || !workspace ||
        q < 1 || q_t < 1 || alpha_t < 1 || rounds_t < 1 || alpha < 1 || rounds < 1)
        return RK_EINVAL;
    const Plan& pa = plan_A->p;
    const Plan& pt = plan_At->p;
    if (pa.dt != RK_F32 || pt.dt != RK_F32 || pt.m != pa.n || pt.n != pa.m || ldg < pa.n)
        return RK_EINVAL;
    if (!aligned16(grad_A) || (ldg * 4) % 16 != 0 || ((uintptr_t)workspace & 255u) != 0)
        return RK_EALIGN;
    rk_opts ot, oa;
    rk_opts_default(&ot);
    rk_opts_default(&oa);
    if (opts_t) ot = *opts_t;
    if (opts) oa = *opts;
    ot.criterion = 0;
    oa.criterion = 0;
    if (!solve_opts_valid(ot, q_t) || !solve_opts_valid(oa, q)) return RK_EINVAL;
    if (ws_bytes < adjoint_ws_bytes(&pa, &pt, q_t, q)) return RK_EWORKSPACE;
    return run_adjoint(&pa, &pt, b, x, gx, q_t, q, alpha_t, rounds_t, alpha, rounds, seed, ot, oa,
                       grad_b, grad_A, ldg, g, workspace, static_cast<cudaStream_t>(stream));
}

size_t rk_solve_residual_workspace_bytes(const rk_plan* plan, int q) {
    if (!plan || q < 1) return 0;
    return align256(solve_ws_bytes(&plan->p, q)) + align256(residual_ws_bytes(plan->p.m, plan->p.n)) +
           256;
}

int rkab_solve_residual(const rk_plan* plan, const float* A32, int64_t lda32, const float* b,
                        const float* x0, float* x, int q, int64_t alpha, int64_t max_rounds,
                        int64_t check_every, uint64_t seed, const rk_opts* opts, int criterion,
                        double tol, void* workspace, size_t ws_bytes, void* stream,
                        int64_t* rounds_done, double* last_metric) {
    if (rounds_done) *rounds_done = 0;
    if (last_metric) *last_metric = -1.0;
    if (!plan || !b || !x0 || !x || !workspace || q < 1 || alpha < 1 || max_rounds < 0 ||
        check_every < 1 || !(tol >= 0.0) || (criterion != RK_CRIT_RESIDUAL && criterion != RK_CRIT_NORMAL))
        return RK_EINVAL;
    const Plan& pl = plan->p;
    if (!A32) {
        if (pl.dt != RK_F32) return RK_EINVAL;
        A32 = static_cast<const float*>(pl.A);
        lda32 = pl.lda;
    }
    if (lda32 < pl.n) return RK_EINVAL;
    if (!aligned16(A32) || (lda32 * 4) % 16 != 0 || ((uintptr_t)workspace & 255u) != 0) return RK_EALIGN;
    rk_opts o;
    rk_opts_default(&o);
    if (opts) o = *opts;
    o.criterion = 0;
    o.check_every = 0;
    o.x_ref = nullptr;
    if (!solve_opts_valid(o, q)) return RK_EINVAL;
    if (ws_bytes < rk_solve_residual_workspace_bytes(plan, q)) return RK_EWORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* p = static_cast<uint8_t*>(workspace);
    SolveInfo* info = reinterpret_cast<SolveInfo*>(p);
    float* V = reinterpret_cast<float*>(p + align256(sizeof(SolveInfo)));
    p += align256(solve_ws_bytes(&pl, q));
    void* rws = p;
    p += align256(residual_ws_bytes(pl.m, pl.n));
    double* norms = reinterpret_cast<double*>(p);
    // ||A||_F^2 = T 2^L from the plan's integer weights (relative truncation below m / T)
    double fro = 0.0;
    if (criterion == RK_CRIT_NORMAL) {
        uint64_t T = 0;
        int32_t L = 0;
        const int rc = rk_plan_status(plan, stream, &T, &L);
        if (rc != RK_OK) return rc;
        fro = std::sqrt(std::ldexp((double)T, L));
    }
    // ||b|| for the relative residual: the residual of x = 0
    double bnorm = 1.0;
    if (criterion == RK_CRIT_RESIDUAL) {
        if (cudaMemsetAsync(x, 0, (size_t)pl.n * 4, st) != cudaSuccess) return RK_ECUDA;
        int rc = launch_residual(A32, pl.m, pl.n, lda32, b, x, nullptr, norms, 0, rws, st);
        double h[2];
        if (rc != RK_OK) return rc;
        if (cudaMemcpyAsync(h, norms, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RK_ECUDA;
        bnorm = h[0] > 0.0 ? h[0] : 1.0;
    }
    const float* start = x0;
    int64_t done = 0;
    while (done < max_rounds) {
        const int64_t k = (max_rounds - done) < check_every ? (max_rounds - done) : check_every;
        SolveArgs a;
        a.plan = &pl;
        a.b = b;
        a.x0 = start;
        a.x = x;
        a.q = q;
        a.alpha = alpha;
        a.rounds = k;
        a.seed = seed;
        a.opts = o;
        a.opts.round0 = o.round0 + done;
        a.info = info;
        a.ldv = (pl.n + 3) / 4 * 4;
        a.V = V;
        if (cudaMemsetAsync(info, 0, sizeof(SolveInfo), st) != cudaSuccess) return RK_ECUDA;
        int rc = launch_solve(a, st);
        if (rc != RK_OK) return rc;
        start = x;
        rc = launch_residual(A32, pl.m, pl.n, lda32, b, x, nullptr, norms, criterion == RK_CRIT_NORMAL,
                             rws, st);
        if (rc != RK_OK) return rc;
        double h[2];
        int status = 0;
        if (cudaMemcpyAsync(h, norms, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&status, &info->status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RK_ECUDA;
        if (status != 0) return status;
        done += k;
        if (rounds_done) *rounds_done = done;
        double metric;
        if (criterion == RK_CRIT_RESIDUAL) metric = h[0] / bnorm;
        else metric = (h[0] > 0.0 && fro > 0.0) ? h[1] / (fro * h[0]) : 0.0;
        if (last_metric) *last_metric = metric;
        if (!std::isfinite(metric)) return RK_EDIVERGED;
        if (metric < tol) break;
    }
    return RK_OK;
}

double rk_alpha_star(int q, double s_min, double s_max) {
    if (q < 1 || !(s_min >= 0.0 && s_min <= 1.0) || !(s_max >= 0.0 && s_max <= 1.0)) return 0.0;
    if (q == 1 || s_max - s_min <= 1.0 / (double)(q - 1)) return (double)q / (1.0 + (q - 1) * s_min);
    return 2.0 * q / (1.0 + (q - 1) * (s_min + s_max));
}

int rk_plan_frobenius2(const rk_plan* plan, void* stream, double* fro2) {
    if (!plan || !fro2) return RK_EINVAL;
    uint64_t T = 0;
    int32_t L = 0;
    const int rc = rk_plan_status(plan, stream, &T, &L);
    if (rc != RK_OK) return rc;
    *fro2 = std::ldexp((double)T, L);   // sum of the integer row weights K_i 2^L
    return RK_OK;
}

int rk_spectrum_ratios(const double* spectrum, double* s_min, double* s_max) {
    if (!spectrum || !(spectrum[2] > 0.0) || !std::isfinite(spectrum[2])) return RK_EINVAL;
    // s = sigma^2 / ||A||_F^2 (Eq. (best_alpha)), clamped to [0, 1] against rounding
    const double lo = std::fmin(std::fmax(spectrum[0] / spectrum[2], 0.0), 1.0);
    const double hi = std::fmin(std::fmax(spectrum[1] / spectrum[2], 0.0), 1.0);
    if (s_min) *s_min = lo;
    if (s_max) *s_max = hi;
    return RK_OK;
}

static int lanczos_steps(int64_t m, int64_t n, int k) {   // at most min(m, n) are of use
    const int64_t r = m < n ? m : n;
    return (int)(k < r ? k : r);
}

size_t rk_spectrum_workspace_bytes(int64_t m, int64_t n, int k) {
    if (m < 1 || n < 1 || k < 1 || k > 512) return 0;
    return spectrum_ws_bytes(m, n, lanczos_steps(m, n, k));
}

int rk_spectrum(const float* A, int64_t m, int64_t n, int64_t lda, int k, uint64_t seed,
                void* workspace, size_t ws_bytes, void* stream, double* out, int* steps_done) {
    if (!A || !workspace || !out || m < 1 || n < 1 || lda < n || k < 1 || k > 512) return RK_EINVAL;
    if (!aligned16(A) || (lda * 4) % 16 != 0 || ((uintptr_t)workspace & 255u) != 0) return RK_EALIGN;
    const int kk = lanczos_steps(m, n, k);
    if (ws_bytes < spectrum_ws_bytes(m, n, kk)) return RK_EWORKSPACE;
    return run_spectrum(A, m, n, lda, kk, seed, workspace, static_cast<cudaStream_t>(stream), out,
                        steps_done);
}

int rk_spectrum_ex(const float* A, int64_t m, int64_t n, int64_t lda, int k, uint64_t seed, double fro2,
                   void* workspace, size_t ws_bytes, void* stream, double* out, int* steps_done) {
    if (!A || !workspace || !out || m < 1 || n < 1 || lda < n || k < 1 || k > 512) return RK_EINVAL;
    if (!aligned16(A) || (lda * 4) % 16 != 0 || ((uintptr_t)workspace & 255u) != 0) return RK_EALIGN;
    if (!std::isfinite(fro2)) return RK_EINVAL;
    const int kk = lanczos_steps(m, n, k);
    if (ws_bytes < spectrum_ws_bytes(m, n, kk)) return RK_EWORKSPACE;
    return run_spectrum(A, m, n, lda, kk, seed, workspace, static_cast<cudaStream_t>(stream), out,
                        steps_done, fro2);
}

int rk_optimal_weight(const float* A, int64_t m, int64_t n, int64_t lda, int q, int k, uint64_t seed,
                      double fro2, void* workspace, size_t ws_bytes, void* stream, double* alpha,
                      double* out, int* steps_done) {
    if (!alpha || q < 1) return RK_EINVAL;
    double sp[3];
    const int rc = rk_spectrum_ex(A, m, n, lda, k, seed, fro2, workspace, ws_bytes, stream, sp, steps_done);
    if (rc != RK_OK) return rc;
    double s_min = 0.0, s_max = 0.0;
    if (rk_spectrum_ratios(sp, &s_min, &s_max) != RK_OK) return RK_EINVAL;   // a zero matrix
    const double a = rk_alpha_star(q, s_min, s_max);
    if (!(a > 0.0)) return RK_EINVAL;
    *alpha = a;
    if (out) {
        out[0] = sp[0];
        out[1] = sp[1];
        out[2] = sp[2];
        out[3] = s_min;
        out[4] = s_max;
    }
    return RK_OK;
}

size_t rk_partial_alpha_workspace_bytes(int64_t m, int64_t n, int q, int k) {
    if (m < 1 || n < 1 || q < 1 || q > m || k < 1 || k > 512) return 0;
    const int64_t rows = (m + q - 1) / q + 1;   // the largest block
    return spectrum_ws_bytes(rows, n, lanczos_steps(rows, n, k));
}

int rk_partial_alpha_star(const float* A, int64_t m, int64_t n, int64_t lda, int q, int k,
                          uint64_t seed, void* workspace, size_t ws_bytes, void* stream,
                          float* weights, double* spectra) {
    if (!A || !workspace || !weights || m < 1 || n < 1 || lda < n || q < 1 || q > m || k < 1 || k > 512)
        return RK_EINVAL;
    if (!aligned16(A) || (lda * 4) % 16 != 0 || ((uintptr_t)workspace & 255u) != 0) return RK_EALIGN;
    if (ws_bytes < rk_partial_alpha_workspace_bytes(m, n, q, k)) return RK_EWORKSPACE;
    for (int g = 0; g < q; ++g) {
        // the Distributed Approach's block of worker g (Section 3.3.1)
        const int64_t lo = (int64_t)g * m / q, hi = (int64_t)(g + 1) * m / q;
        double out[3];
        const int rc = run_spectrum(A + lo * lda, hi - lo, n, lda, lanczos_steps(hi - lo, n, k), seed,
                                    workspace, static_cast<cudaStream_t>(stream), out, nullptr);
        if (rc != RK_OK) return rc;
        double s_min = 0.0, s_max = 0.0;
        if (rk_spectrum_ratios(out, &s_min, &s_max) != RK_OK) return RK_EINVAL;   // a zero block has no law
        weights[g] = (float)rk_alpha_star(q, s_min, s_max);
        if (spectra) {
            spectra[3 * g] = out[0];
            spectra[3 * g + 1] = out[1];
            spectra[3 * g + 2] = out[2];
        }
    }
    return RK_OK;
}

size_t rk_residual_workspace_bytes(int64_t m, int64_t n) {
    if (m < 1 || n < 1) return 0;
    return residual_ws_bytes(m, n);
}

int rk_residual(const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
                const float* x, double* r, double* norms_out, int want_atr, void* workspace,
                size_t ws_bytes, void* stream) {
    if (!A || !b || !x || !workspace || m < 1 || n < 1 || lda < n) return RK_EINVAL;
    if (!aligned16(A) || (lda * 4) % 16 != 0 || ((uintptr_t)workspace & 255u) != 0)
        return RK_EALIGN;
    if (ws_bytes < residual_ws_bytes(m, n)) return RK_EWORKSPACE;
    return launch_residual(A, m, n, lda, b, x, r, norms_out, want_atr, workspace,
                           static_cast<cudaStream_t>(stream));
}

}  // extern "C"
