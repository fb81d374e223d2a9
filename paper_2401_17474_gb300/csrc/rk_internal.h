// rk_internal.h -- layouts of the device workspaces and the launchers the
// C-ABI layer (rk_api.cu) calls.  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rkab.h"

namespace rk {

typedef unsigned __int128 u128;

constexpr int kNoRows = -(1 << 30);  // H before any nonzero row was seen

// Device-side results of the setup (first 256 bytes of the setup workspace).
struct SetupInfo {
    int status;      // 0, or RK_EINVAL for non-finite / all-zero A
    int H;           // max_i bitlength(R_i) + 2 e_i - 102
    int L;           // H + ceil(log2 m) - 62
    int pad0;
    uint64_t T;      // sum_i K_i
    uint32_t nl, nh; // number of light / heavy buckets
    uint32_t range_rows;  // nonzero rows with ||A_i||^2 outside [2^-126, 2^126): no float32
                          // reciprocal (inv_i = 0); never drawn when the plan succeeds
    uint32_t pad1;
};

// Pointers into the setup workspace.  The first group is the plan's tables
// (kept for the solves); the rest is scratch of the build.
struct SetupWs {
    SetupInfo* info;
    uint64_t* K;
    uint64_t* P;
    uint64_t* thr64;
    uint32_t* alias;
    float* inv;
    // scratch
    u128* R;
    int* e;
    uint32_t* row_pos;
    u128* row_Dex;
    u128* light_Dinc;
    u128* heavy_Einc;
    uint32_t* heavy_idx;
    void* tiles;
    void* tile_total;
};

size_t setup_ws_bytes(int64_t m);
SetupWs setup_ws_carve(void* base, int64_t m);
size_t scan_tiles_bytes(int64_t m);
size_t scan_item_bytes();

int launch_setup(const void* A, rk_dtype dt, const float* row_scale, int64_t m, int64_t n,
                 int64_t lda, const SetupWs& ws, cudaStream_t st);

// Device-side results of a solve (first 256 bytes of the solve workspace).
struct SolveInfo {
    int status;
    int pad0;
    int64_t rounds_done;
    double last_metric;
    unsigned long long bar_arrivals;   // monotonic arrival count of grid_sync
};

struct Plan {
    const void* A;
    rk_dtype dt;
    const float* row_scale;
    int64_t m, n, lda;
    SetupWs ws;
};

struct SolveArgs {
    const Plan* plan;
    const float* b;
    const float* x0;
    float* x;
    int q;
    int64_t alpha;
    int64_t rounds;
    uint64_t seed;
    rk_opts opts;
    SolveInfo* info;
    float* V;          // q x ldv floats (the workers' iterates before the average)
    int64_t ldv;
};

int launch_sample_indices_ex(const Plan* plan, uint64_t seed, uint32_t worker, uint32_t q,
                             uint32_t stream_id, int sampling, uint64_t t0, int64_t count,
                             uint32_t* out, cudaStream_t st);
int v_rows(int q);
int v_rows_for(int q, int64_t alpha);
size_t solve_ws_bytes(const Plan* plan, int q);                        // any alpha
size_t solve_ws_bytes_for(const Plan* plan, int q, int64_t alpha);     // what (q, alpha) uses
bool sampling_ok(const rk_opts& o);
bool solve_opts_valid(const rk_opts& o, int q);                        // the solves' option checks
int launch_solve(const SolveArgs& a, cudaStream_t st);
// RKA (alpha = 1) on rows too long for one CTA: x split by columns over the grid,
// up to 64 workers a round
inline bool colsplit_fits(int64_t alpha, int q) { return alpha == 1 && q >= 1 && q <= 64; }
int launch_sample_indices(const Plan* plan, uint64_t seed, uint32_t worker, uint32_t stream_id,
                          uint64_t t0, int64_t count, uint32_t* out, cudaStream_t st);

size_t residual_ws_bytes(int64_t m, int64_t n);
int launch_residual(const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
                    const float* x, double* r, double* norms_out, int want_atr, void* ws,
                    cudaStream_t st);

int launch_normal_matvec(const float* A, int64_t m, int64_t n, int64_t lda, const float* v,
                         double* w, void* ws, cudaStream_t st);
int launch_rows_matvec(const float* A, int64_t m, int64_t n, int64_t lda, const float* v, double* r,
                       void* ws, cudaStream_t st);
int launch_transpose_matvec(const float* A, int64_t m, int64_t n, int64_t lda, const double* u,
                            double* w, void* ws, cudaStream_t st);
size_t spectrum_ws_bytes(int64_t m, int64_t n, int k);
int run_spectrum(const float* A, int64_t m, int64_t n, int64_t lda, int k, uint64_t seed, void* ws,
                 cudaStream_t st, double* out, int* steps_done, double fro2_known = 0.0);

int launch_quantize(const float* A, int64_t m, int64_t n, int64_t lda, rk_dtype dt, void* out,
                    int64_t ldo, float* row_scale, cudaStream_t st);
size_t refine_ws_bytes(const Plan* pl, int q);
int run_refine(const Plan* lowp, const float* A32, int64_t lda32, const float* b, const float* x0,
               float* x, int q, int64_t alpha, int64_t inner_rounds, int64_t max_outer,
               uint64_t seed, const rk_opts& o, void* ws, cudaStream_t st, int64_t* outer_done,
               double* last_metric);

int launch_transpose(const float* A, int64_t m, int64_t n, int64_t lda, float* At, int64_t ldt,
                     cudaStream_t st);
int launch_rank2(const float* r, const float* g, const float* y, const float* x, int64_t m, int64_t n,
                 float* G, int64_t ldg, cudaStream_t st);
size_t adjoint_ws_bytes(const Plan* pa, const Plan* pt, int q_t, int q);
int run_adjoint(const Plan* pa, const Plan* pt, const float* b, const float* x, const float* gx,
                int q_t, int q, int64_t alpha_t, int64_t rounds_t, int64_t alpha, int64_t rounds, uint64_t seed,
                const rk_opts& ot, const rk_opts& oa, float* grad_b, float* grad_A, int64_t ldg,
                float* g_out, void* ws, cudaStream_t st);

void count_launch(int k = 1);

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Relaxation / uniform row weight of Eqs. (alg) and (rka_eq): positive and below
// 2q.  A single chain (q = 1) converges for omega in (0, 2); the averaged step of
// q projections from one point tolerates weights up to the optimum of
// Eq. (best_alpha), which lies in (0, 2q).
inline bool omega_ok(float omega, int q) {
    return omega > 0.0f && omega < 2.0f * (float)(q < 1 ? 1 : q);
}

}  // namespace rk

// The opaque handle of rkab.h: a host-side Plan.
struct rk_plan {
    rk::Plan p;
};
