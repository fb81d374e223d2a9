// rk_noalloc.cu -- rkab_solve_noalloc: the RKAB solve for callers that cannot
// allocate device memory at all.
//
// Who needs it: code that runs where device allocation is not available to
// it -- a plugin or callback hosted by another runtime that owns every device
// allocation and hands out only a stream, or a real-time control loop that
// forbids allocation once it has started.  Such a caller cannot size and pass
// the solve workspace that rkab_solve takes, so this entry point keeps that
// scratch (the run-state header, the q x n block of worker displacements and
// the averaged iterate) in one fixed file-scope device array instead.
//
// The array is RK_NOALLOC_SCRATCH_BYTES bytes and lives in the library's
// device image: every GPU that loads the library holds it until the process
// exits.  Host code cannot use the array's name as a device address (on the
// host it is only a stand-in symbol), so the address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device; that first call should therefore come before any
// stream capture.  All calls on a device share the array and it keeps the last
// call's contents: the run-state header is cleared by every call, and calls
// whose work overlaps on the GPU race on the array.  The looked-up address is
// cached for the life of the process: it does not survive cudaDeviceReset (or
// any other teardown of the device's primary context), after which this entry
// point must not be called.
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "rk_internal.h"

namespace rk {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RK_NOALLOC_SCRATCH_BYTES];

static constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device (looked up once per device).
static int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RK_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RK_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RK_OK;
}

}  // namespace rk

using namespace rk;

extern "C" int rkab_solve_noalloc(const rk_plan* plan, const float* b, const float* x0, float* x,
                                  int q, int64_t alpha, int64_t rounds, uint64_t seed,
                                  const rk_opts* opts, rk_solve_result* result, void* stream) {
    if (!plan || !b || !x0 || !x || q < 1 || alpha < 1 || rounds < 0) return RK_EINVAL;
    rk_opts o;
    rk_opts_default(&o);
    if (opts) o = *opts;
    if (!solve_opts_valid(o, q)) return RK_EINVAL;   // the checks of rkab_solve
    // the layout of the rkab_solve workspace, with the rows of V this launch uses (one
    // per SM for RKA with more workers than SMs), must fit the fixed array
    if (solve_ws_bytes_for(&plan->p, q, alpha) > (size_t)RK_NOALLOC_SCRATCH_BYTES) return RK_ETOOLARGE;
    void* scratch = nullptr;
    const int rc0 = scratch_address(&scratch);
    if (rc0 != RK_OK) return rc0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SolveInfo* info = static_cast<SolveInfo*>(scratch);
    if (cudaMemsetAsync(info, 0, sizeof(SolveInfo), st) != cudaSuccess) return RK_ECUDA;
    int rc = RK_OK;
    if (rounds == 0) {
        if (x != x0 &&
            cudaMemcpyAsync(x, x0, (size_t)plan->p.n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = RK_ECUDA;
    } else {
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
        a.ldv = (plan->p.n + 3) / 4 * 4;
        a.V = reinterpret_cast<float*>(static_cast<unsigned char*>(scratch) + align256(sizeof(SolveInfo)));
        rc = launch_solve(a, st);
    }
    if (rc == RK_OK && result) {
        static_assert(offsetof(SolveInfo, status) == offsetof(rk_solve_result, status), "layout");
        static_assert(offsetof(SolveInfo, rounds_done) == offsetof(rk_solve_result, rounds_done), "layout");
        static_assert(offsetof(SolveInfo, last_metric) == offsetof(rk_solve_result, last_metric), "layout");
        if (cudaMemcpyAsync(result, info, sizeof(rk_solve_result), cudaMemcpyDefault, st) != cudaSuccess)
            rc = RK_ECUDA;
    }
    return rc;
}
