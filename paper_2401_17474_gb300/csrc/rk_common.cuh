// rk_common.cuh -- device helpers shared by the library's kernels:
// Philox4x32-10, the row sampler, PTX wrappers for mbarriers and bulk
// asynchronous copies, the device clock, and a grid barrier whose waits are
// bounded in time.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rkab.h"

namespace rk {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3" (SC'11).  Each round multiplies words 0 and 2 by the two round
// multipliers, mixes the high halves with words 1 and 3 and the round key;
// the key advances by the two Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Draw of (seed, worker, t, stream): bucket from the first 64 random bits, side
// of the bucket from the second 64 (see rk_sample_indices in rkab.h).
__device__ __forceinline__ uint32_t sample_row(uint64_t seed, uint32_t worker, uint32_t stream,
                                               uint64_t t, uint64_t m,
                                               const uint64_t* __restrict__ thr64,
                                               const uint32_t* __restrict__ alias) {
    const U4 r = philox10(U4{(uint32_t)t, (uint32_t)(t >> 32), worker, stream},
                          (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t u = (uint64_t)r.x | ((uint64_t)r.y << 32);
    const uint64_t u2 = (uint64_t)r.z | ((uint64_t)r.w << 32);
    const uint64_t c = __umul64hi(u, m);
    const uint64_t th = __ldg(thr64 + c);
    return u2 < th ? (uint32_t)c : __ldg(alias + c);
}

// ---------------------------------------------------------------------------
// Clock and bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_status(int* status, int code) {
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Limit of the wait for a CTA's own bulk copies in flight before it exits: at
// least 2 s whatever the caller's limit, since a copy that was issued completes
// in microseconds and the CTA must not exit while one is still writing its
// shared memory.
__device__ __forceinline__ uint64_t drain_limit_ns(uint64_t timeout_ns) {
    return timeout_ns > 2000000000ull ? timeout_ns : 2000000000ull;
}

// Grid-wide barrier on a monotonic arrival counter (zero at launch): the b-th
// barrier of every CTA (b = 0, 1, ...) completes when the counter reaches
// (b + 1) * nblocks, so no CTA resets anything and the last arriver's single
// atomic releases everyone.  Called by ONE thread per CTA, after a CTA-wide
// barrier, with its own count b of barriers passed: the acq_rel atomic publishes
// the CTA's writes (release is cumulative over what the CTA barrier ordered
// before it) and the acquire load of the waiters orders their later reads.
// Returns false (leaving an error in *status) when the wait exceeds timeout_ns
// or another CTA has already failed; a CTA that failed never arrives, so the
// others find its status in their spins.
__device__ __forceinline__ bool grid_sync(unsigned long long* count, unsigned long long b,
                                          unsigned nblocks, int* status, uint64_t timeout_ns) {
    const unsigned long long target = (b + 1ull) * (unsigned long long)nblocks;
    unsigned long long prev;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], 1;" : "=l"(prev) : "l"(count) : "memory");
    if (prev + 1ull >= target) return true;
    uint64_t t0 = 0;
    for (unsigned spins = 1;; ++spins) {
        if (ld_acquire_gpu_u64(count) >= target) return true;
        if ((spins & 63u) == 0) {
            if (ld_acquire_gpu(status) != 0) return false;
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > timeout_ns) {
                set_status(status, RK_ETIMEOUT);
                return false;
            }
        }
        if (spins > 256) __nanosleep(32);
    }
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy wrappers (PTX ISA: mbarrier.*, cp.async.bulk).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing tx bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace rk
