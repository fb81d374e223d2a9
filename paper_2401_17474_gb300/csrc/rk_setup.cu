// rk_setup.cu -- sampling tables of Eq. (prob_line) (Section 2.2) on the GPU:
// exact integer row weights K_i, their exclusive prefix P_i and total T, the
// alias table of the law K_i / T (sweeping construction, computed in parallel
// from prefix sums of the lights' deficits and the heavies' excesses), and the
// float32 reciprocals 1/||A_i||^2 of the projection of Eq. (alg).
//
// Every integer here is exact, so the tables do not depend on the order in
// which threads add; they equal, bit for bit, those of any implementation of
// the definitions in rkab.h.
#include <cstdint>
#include <cstdio>

#include "rk_common.cuh"
#include "rk_internal.h"

namespace rk {

// ---------------------------------------------------------------------------
// Element loaders: 16-byte chunks of a row decoded to float32.
// ---------------------------------------------------------------------------
struct LoadF32 {
    static constexpr int kPerChunk = 4;
    static constexpr int kBytes = 4;
    __device__ static void decode(const uint4& c, float s, float* out) {
        (void)s;
        out[0] = __uint_as_float(c.x);
        out[1] = __uint_as_float(c.y);
        out[2] = __uint_as_float(c.z);
        out[3] = __uint_as_float(c.w);
    }
    // float32 bits of the largest |decoded value| of the chunk
    __device__ static uint32_t max_abs_bits(const uint4& c, float s) {
        (void)s;
        return max(max(c.x & 0x7FFFFFFFu, c.y & 0x7FFFFFFFu), max(c.z & 0x7FFFFFFFu, c.w & 0x7FFFFFFFu));
    }
};

struct LoadBF16 {
    static constexpr int kPerChunk = 8;
    static constexpr int kBytes = 2;
    __device__ static void decode(const uint4& c, float s, float* out) {
        (void)s;
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            out[2 * k] = __uint_as_float(w[k] << 16);
            out[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
    __device__ static uint32_t max_abs_bits(const uint4& c, float s) {
        (void)s;
        const uint32_t h = __vmaxu2(__vmaxu2(c.x & 0x7FFF7FFFu, c.y & 0x7FFF7FFFu),
                                    __vmaxu2(c.z & 0x7FFF7FFFu, c.w & 0x7FFF7FFFu));
        return max(h & 0xFFFFu, h >> 16) << 16;
    }
};

// OCP FP8 e4m3, finite-only variant: 1 sign, 4 exponent (bias 7), 3 mantissa bits.
__device__ __forceinline__ float e4m3_to_float(uint32_t code) {
    const uint32_t sgn = (code & 0x80u) << 24;
    const uint32_t e = (code >> 3) & 0xFu;
    const uint32_t f = code & 7u;
    float v;
    if (e == 0) {
        v = (float)f * 0.001953125f;  // f / 8 * 2^-6 = f * 2^-9, exact
    } else {
        v = __uint_as_float(((e + 120u) << 23) | (f << 20));  // (1 + f/8) 2^(e-7)
    }
    return __uint_as_float(__float_as_uint(v) | sgn);
}

struct LoadFP8 {
    static constexpr int kPerChunk = 16;
    static constexpr int kBytes = 1;
    __device__ static void decode(const uint4& c, float s, float* out) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int b = 0; b < 4; ++b) out[4 * k + b] = __fmul_rn(s, e4m3_to_float((w[k] >> (8 * b)) & 0xFFu));
        }
    }
    // e4m3 decoding is increasing in the 7-bit magnitude code and rounding is
    // monotone and sign-symmetric, so the largest |s q| is |s| times the
    // largest magnitude code's value
    __device__ static uint32_t max_abs_bits(const uint4& c, float s) {
        const uint32_t b = __vmaxu4(__vmaxu4(c.x & 0x7F7F7F7Fu, c.y & 0x7F7F7F7Fu),
                                    __vmaxu4(c.z & 0x7F7F7F7Fu, c.w & 0x7F7F7F7Fu));
        const uint32_t code = max(max(b & 0xFFu, (b >> 8) & 0xFFu), max((b >> 16) & 0xFFu, b >> 24));
        return __float_as_uint(__fmul_rn(s, e4m3_to_float(code))) & 0x7FFFFFFFu;
    }
};

// ---------------------------------------------------------------------------
// Row weights: R_i = sum_j floor(a_ij^2 2^(102 - 2 e_i)) exactly, e_i the
// frexp exponent of max_j |a_ij|; h_i = bitlength(R_i) + 2 e_i - 102 (max -> H).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int frexp_exp_of_absbits(uint32_t ab) {
    const uint32_t E = ab >> 23;
    if (E != 0) return (int)E - 126;
    return (32 - __clz(ab)) - 149;  // subnormal: M 2^-149 with M in [2^(bl-1), 2^bl)
}

// Exact sum of floor(a^2 2^(102 - 2 e)) over entries with |a| < 2^e.  For an
// entry mant 2^(E - 150) (E = 1 for a subnormal, without the implicit bit),
// U = |a| 2^(51 - e) = mant 2^k with k = E - 99 - e.  When k >= 0, U is an
// integer below 2^51 and the term is U^2 = Uh^2 2^54 + Uh Ul 2^28 + Ul^2 with
// U = Uh 2^27 + Ul, so three 32 x 32 -> 64-bit multiply-adds take it exactly
// (each sum below 2^63 for up to 512 entries).  When k < 0 the term is
// floor(mant^2 2^(2k)).
//
// SqAcc is for rows with e >= -90, where k <= 27 and every zero or subnormal
// entry has k < 0: add() takes the k >= 0 terms with 32-bit funnel shifts
// (Uh = mant >> (27 - k), Ul = (mant << k) mod 2^27; both clamp to 0 when
// k < 0) and tracks the smallest nonzero |a|; when that lies below 2^(kbase-127)
// (some entry has k < 0) add_small() adds the k < 0 terms.  SqAccWide takes
// any row.
// acc += a * b (32 x 32 -> 64 bits) as one multiply-add
__device__ __forceinline__ void mad_wide(uint64_t& acc, uint32_t a, uint32_t b) {
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

struct SqAcc {
    uint64_t hh = 0, hl = 0, ll = 0, tiny = 0;
    uint32_t minab = 0xFFFFFFFFu;   // min over entries of |a| bits - 1 (a zero wraps to the top)
    __device__ __forceinline__ void add(uint32_t ab, uint32_t kbase) {   // kbase = 99 + e
        const uint32_t E = ab >> 23;
        const uint32_t mant = (ab & 0x7FFFFFu) | 0x800000u;   // E = 0 has k < 0: no term here
        const uint32_t uh = __funnelshift_rc(mant, 0u, kbase + 27u - E);
        const uint32_t ul = __funnelshift_lc(0u, mant, E - kbase) & 0x7FFFFFFu;
        mad_wide(hh, uh, uh);
        mad_wide(hl, uh, ul);
        mad_wide(ll, ul, ul);
        minab = min(minab, ab - 1u);
    }
    __device__ __forceinline__ bool has_small(uint32_t kbase) const { return minab < (kbase << 23) - 1u; }
    __device__ __forceinline__ void add_small(uint32_t ab, uint32_t kbase) {   // the k < 0 terms only
        const uint32_t E = ab >> 23;
        const uint32_t Ee = max(E, 1u);
        const uint32_t mant = ab - ((Ee - 1u) << 23);
        const int k = (int)Ee - (int)kbase;
        if (k < 0 && k > -24) tiny += ((uint64_t)mant * mant) >> (-2 * k);
    }
    __device__ __forceinline__ u128 sums() const { return ((u128)hh << 54) + ((u128)hl << 28) + (u128)ll; }
    __device__ __forceinline__ void clear_sums() { hh = hl = ll = 0; }
};

struct SqAccWide {
    u128 acc = 0;
    __device__ __forceinline__ void add(uint32_t ab, int kbase) {   // kbase = 99 + e
        const uint32_t E = ab >> 23;
        const uint32_t Ee = max(E, 1u);
        const uint32_t mant = ab - ((Ee - 1u) << 23);
        const int k = (int)Ee - kbase;
        if (k >= 0) {
            const u128 U = (u128)mant << k;   // below 2^51
            acc += U * U;
        } else if (k > -24) {
            acc += ((uint64_t)mant * mant) >> (-2 * k);
        }
    }
};

__device__ __forceinline__ int bitlen128(u128 v) {
    const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    if (hi) return 128 - __clzll((long long)hi);
    if (lo) return 64 - __clzll((long long)lo);
    return 0;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int lane_mask) {
    const uint64_t hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), lane_mask);
    const uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, lane_mask);
    return ((u128)hi << 64) | lo;
}

// One warp per row (warp-level reductions only): pass 1 finds max |a| as the
// integer order of the absolute bit patterns, pass 2 forms the exact sum of the
// scaled squares (integer, so its order does not matter; the row is then L1/L2
// resident).  Non-finite rows set RK_EINVAL; zero rows get zero entries.
template <class LD>
__global__ void __launch_bounds__(256) row_weight_kernel(const uint8_t* __restrict__ A,
                                                         const float* __restrict__ row_scale,
                                                         int64_t m, int64_t n, int64_t lda_bytes,
                                                         SetupWs ws) {
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (n + LD::kPerChunk - 1) / LD::kPerChunk;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < m; i += (int64_t)gridDim.x * wpb) {
        const uint4* row = reinterpret_cast<const uint4*>(A + i * lda_bytes);
        const float sc = row_scale ? __ldg(row_scale + i) : 1.0f;
        uint32_t mx = 0;
#pragma unroll 4
        for (int64_t c = lane; c < nchunks; c += 32) {
            float v[LD::kPerChunk];
            LD::decode(__ldg(row + c), sc, v);
#pragma unroll
            for (int k = 0; k < LD::kPerChunk; ++k) {
                if (c * LD::kPerChunk + k < n) mx = max(mx, __float_as_uint(v[k]) & 0x7FFFFFFFu);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (mx >= 0x7F800000u || mx == 0) {  // inf or nan: no law; zero row: weight 0
            if (lane == 0) {
                if (mx != 0) atomicCAS(&ws.info->status, 0, RK_EINVAL);
                ws.R[i] = 0;
                ws.e[i] = 0;
            }
            continue;
        }
        const int e = frexp_exp_of_absbits(mx);
        u128 acc = 0;
        if (e >= -90) {
            const uint32_t kbase = (uint32_t)(99 + e);
            SqAcc sa;
            int since = 0;   // chunks in the sums since they were folded into acc (at most 32: 512 entries)
#pragma unroll 4
            for (int64_t c = lane; c < nchunks; c += 32) {
                float v[LD::kPerChunk];
                LD::decode(__ldg(row + c), sc, v);
#pragma unroll
                for (int k = 0; k < LD::kPerChunk; ++k)
                    if (c * LD::kPerChunk + k < n) sa.add(__float_as_uint(v[k]) & 0x7FFFFFFFu, kbase);
                if (++since == 32) {
                    acc += sa.sums();
                    sa.clear_sums();
                    since = 0;
                }
            }
            if (sa.has_small(kbase)) {   // entries far below the largest: their floors (rare)
                for (int64_t c = lane; c < nchunks; c += 32) {
                    float v[LD::kPerChunk];
                    LD::decode(__ldg(row + c), sc, v);
#pragma unroll
                    for (int k = 0; k < LD::kPerChunk; ++k)
                        if (c * LD::kPerChunk + k < n) sa.add_small(__float_as_uint(v[k]) & 0x7FFFFFFFu, kbase);
                }
            }
            acc += sa.sums() + (u128)sa.tiny;
        } else {   // the largest entry is below 2^-91
            SqAccWide sw;
            for (int64_t c = lane; c < nchunks; c += 32) {
                float v[LD::kPerChunk];
                LD::decode(__ldg(row + c), sc, v);
#pragma unroll
                for (int k = 0; k < LD::kPerChunk; ++k)
                    if (c * LD::kPerChunk + k < n) sw.add(__float_as_uint(v[k]) & 0x7FFFFFFFu, 99 + e);
            }
            acc = sw.acc;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += shfl_xor_u128(acc, o);
        if (lane == 0) {
            ws.R[i] = acc;
            ws.e[i] = e;
            atomicMax(&ws.info->H, bitlen128(acc) + 2 * e - 102);
        }
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The same weights with one CTA per row and S rows of the CTA (rows blockIdx.x,
// + gridDim.x, ...) in flight: every thread copies its own 16-byte chunks (tid,
// tid + NT, ...) of a row into a shared-memory stage with cp.async and reads
// back only those chunks, so the ring needs no barrier and no wait on another
// thread.  The two passes (max |a|, then the exact sum) read the stage, so A is
// read from DRAM once.  Bytes past n in the last chunk are zeroed before
// decoding.
template <class LD, int NT, int S>
__global__ void __launch_bounds__(NT) row_weight_staged_kernel(const uint8_t* __restrict__ A,
                                                               const float* __restrict__ row_scale,
                                                               int64_t m, int64_t n, int64_t lda_bytes,
                                                               SetupWs ws) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) uint4 stage[];
    __shared__ uint32_t s_max[2][NW];
    __shared__ uint64_t s_hi[2][NW], s_lo[2][NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nchunks = (int)((n + LD::kPerChunk - 1) / LD::kPerChunk);
    const int tail_bytes = (int)(n % LD::kPerChunk) * LD::kBytes;   // 0: the last chunk is full
    const bool owns_tail = tail_bytes && tid < nchunks && (nchunks - 1 - tid) % NT == 0;
    const int64_t G = gridDim.x;
    const int64_t J = (m - 1 - blockIdx.x) / G + 1;   // rows of this CTA (gridDim.x <= m)
    auto issue = [&](int64_t j) {
        if (j < J) {
            const uint4* src = reinterpret_cast<const uint4*>(A + (blockIdx.x + j * G) * lda_bytes);
            uint4* dst = stage + (size_t)(j % S) * nchunks;
            for (int idx = tid; idx < nchunks; idx += NT) cp_async16(dst + idx, src + idx);
        }
        cp_async_commit();   // one group a row (empty past the last row)
    };
#pragma unroll
    for (int j = 0; j < S - 1; ++j) issue(j);
    int par = 0;
    for (int64_t j = 0; j < J; ++j, par ^= 1) {
        issue(j + S - 1);         // into the stage this thread finished reading in iteration j - 1
        cp_async_wait<S - 1>();   // this thread's chunks of row j have landed
        const int64_t i = blockIdx.x + j * G;
        uint4* row = stage + (size_t)(j % S) * nchunks;
        const float sc = row_scale ? __ldg(row_scale + i) : 1.0f;
        if (owns_tail) {
            const uint4 c = row[nchunks - 1];
            uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int keep = tail_bytes - 4 * q;   // bytes of word q that lie inside the row
                if (keep <= 0) w[q] = 0u;
                else if (keep < 4) w[q] &= (1u << (8 * keep)) - 1u;
            }
            row[nchunks - 1] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        uint32_t mx = 0;
#pragma unroll 4
        for (int idx = tid; idx < nchunks; idx += NT) mx = max(mx, LD::max_abs_bits(row[idx], sc));
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_max[par][wid] = mx;
        __syncthreads();
        mx = s_max[par][0];
#pragma unroll
        for (int w = 1; w < NW; ++w) mx = max(mx, s_max[par][w]);
        if (mx >= 0x7F800000u || mx == 0) {  // inf or nan: no law; zero row: weight 0
            if (tid == 0) {
                if (mx != 0) atomicCAS(&ws.info->status, 0, RK_EINVAL);
                ws.R[i] = 0;
                ws.e[i] = 0;
            }
            continue;
        }
        const int e = frexp_exp_of_absbits(mx);
        u128 mine;
        if (e >= -90) {
            const uint32_t kbase = (uint32_t)(99 + e);
            SqAcc sa;   // at most 16 entries a chunk and 16 chunks a thread: 256 entries
#pragma unroll 4
            for (int idx = tid; idx < nchunks; idx += NT) {
                float v[LD::kPerChunk];
                LD::decode(row[idx], sc, v);
#pragma unroll
                for (int q = 0; q < LD::kPerChunk; ++q) sa.add(__float_as_uint(v[q]) & 0x7FFFFFFFu, kbase);
            }
            if (sa.has_small(kbase)) {   // entries far below the largest: their floors (rare)
                for (int idx = tid; idx < nchunks; idx += NT) {
                    float v[LD::kPerChunk];
                    LD::decode(row[idx], sc, v);
#pragma unroll
                    for (int q = 0; q < LD::kPerChunk; ++q)
                        sa.add_small(__float_as_uint(v[q]) & 0x7FFFFFFFu, kbase);
                }
            }
            mine = sa.sums() + (u128)sa.tiny;
        } else {   // the largest entry is below 2^-91
            SqAccWide sw;
            for (int idx = tid; idx < nchunks; idx += NT) {
                float v[LD::kPerChunk];
                LD::decode(row[idx], sc, v);
#pragma unroll
                for (int q = 0; q < LD::kPerChunk; ++q) sw.add(__float_as_uint(v[q]) & 0x7FFFFFFFu, 99 + e);
            }
            mine = sw.acc;
        }
        uint64_t hi = (uint64_t)(mine >> 64), lo = (uint64_t)mine;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const uint64_t ol = __shfl_xor_sync(0xffffffffu, (unsigned long long)lo, o);
            const uint64_t oh = __shfl_xor_sync(0xffffffffu, (unsigned long long)hi, o);
            lo += ol;
            hi += oh + (lo < ol ? 1ull : 0ull);
        }
        if (lane == 0) {
            s_hi[par][wid] = hi;
            s_lo[par][wid] = lo;
        }
        __syncthreads();
        if (tid == 0) {
            u128 acc = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) acc += ((u128)s_hi[par][w] << 64) | s_lo[par][w];
            ws.R[i] = acc;
            ws.e[i] = e;
            atomicMax(&ws.info->H, bitlen128(acc) + 2 * e - 102);
        }
    }
    cp_async_wait<0>();
}

// K_i = R_i >> (L + 102 - 2 e_i); L = H + ceil(log2 m) - 62; and
// inv_i = 1 / ||A_i||^2 in float32; 0 for a zero row and for a row whose ||A_i||^2 lies
// outside [2^-126, 2^126) (counted in range_rows; the plan fails if the law can draw it).
__global__ void weights_to_k_kernel(int64_t m, SetupWs ws) {
    const int H = ws.info->H;
    if (H == kNoRows) {  // all rows zero: no law
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&ws.info->status, 0, RK_EINVAL);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
             i += (int64_t)gridDim.x * blockDim.x) {
            ws.K[i] = 0;
            ws.inv[i] = 0.0f;
        }
        return;
    }
    int c = 0;
    while (((int64_t)1 << c) < m) ++c;
    const int L = H + c - 62;
    if (blockIdx.x == 0 && threadIdx.x == 0) ws.info->L = L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const u128 R = ws.R[i];
        uint64_t K = 0;
        float inv = 0.0f;
        if (R != 0) {
            const int e = ws.e[i];
            const int sh = L + 102 - 2 * e;
            K = (sh >= 128) ? 0 : (uint64_t)(R >> sh);  // sh >= 0 by construction of L
            // 1 / ||A_i||^2 with ||A_i||^2 = R 2^(2e - 102) (R rounded to double once)
            const double rd = (double)(uint64_t)(R >> 64) * 18446744073709551616.0 + (double)(uint64_t)R;
            const double w = ldexp(rd, 2 * e - 102);
            if (w >= 0x1p-126 && w < 0x1p126) {
                inv = (float)(1.0 / w);
            } else {
                // outside the float32 range of the projection: 1/||A_i||^2 would overflow
                // (or underflow), and the row's products with x underflow; the solve
                // cannot project on such a row, so a plan that can draw one fails
                atomicAdd(&ws.info->range_rows, 1u);
                if (K != 0) atomicCAS(&ws.info->status, 0, RK_EINVAL);
            }
        }
        ws.K[i] = K;
        ws.inv[i] = inv;
    }
}

// ---------------------------------------------------------------------------
// Exact device-wide exclusive scans over rows (three passes: tile totals, one
// block over the tile totals, tile rescans).  Integer addition is associative,
// so the result is the same for any decomposition.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanIpt = 4;
constexpr int kScanTile = kScanThreads * kScanIpt;

struct ItemK {
    uint64_t k;
    __device__ ItemK operator+(const ItemK& o) const { return ItemK{k + o.k}; }
};

struct ItemC {  // classification: counts of lights / heavies, deficit D and excess E
    uint32_t nl, nh;
    u128 D, E;
    __device__ ItemC operator+(const ItemC& o) const { return ItemC{nl + o.nl, nh + o.nh, D + o.D, E + o.E}; }
};

struct GetK {
    const uint64_t* K;
    __device__ ItemK operator()(int64_t i) const { return ItemK{K[i]}; }
};

struct PutK {
    uint64_t* P;
    __device__ void operator()(int64_t i, const ItemK& excl, const ItemK& own) const {
        (void)own;
        P[i] = excl.k;
    }
};

__device__ __forceinline__ ItemC classify(const uint64_t* K, int64_t i, uint64_t m, uint64_t T) {
    const u128 S = (u128)m * (u128)K[i];
    const u128 TT = (u128)T;
    if (S < TT) return ItemC{1u, 0u, TT - S, 0};
    if (S > TT) return ItemC{0u, 1u, 0, S - TT};
    return ItemC{0u, 0u, 0, 0};
}

struct GetC {
    const uint64_t* K;
    uint64_t m;
    const SetupInfo* info;
    __device__ ItemC operator()(int64_t i) const { return classify(K, i, m, info->T); }
};

// Compaction: light k -> its inclusive deficit prefix; heavy p -> its row and inclusive excess.
struct PutC {
    SetupWs ws;
    __device__ void operator()(int64_t i, const ItemC& excl, const ItemC& own) const {
        if (own.nl) {
            ws.light_Dinc[excl.nl] = excl.D + own.D;
            ws.row_pos[i] = excl.nl;
            ws.row_Dex[i] = excl.D;
        } else if (own.nh) {
            ws.heavy_idx[excl.nh] = (uint32_t)i;
            ws.heavy_Einc[excl.nh] = excl.E + own.E;
            ws.row_pos[i] = excl.nh;
        }
    }
};

template <class Item>
__device__ Item block_exclusive_scan(Item v, Item* sm, Item& total) {
    // Hillis-Steele inclusive scan in shared memory, then shift.
    const int t = threadIdx.x;
    sm[t] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        Item add = v;
        const bool has = t >= off;
        if (has) add = sm[t - off];
        __syncthreads();
        if (has) v = add + v;
        sm[t] = v;
        __syncthreads();
    }
    total = sm[blockDim.x - 1];
    Item ex = (t > 0) ? sm[t - 1] : Item{};
    __syncthreads();
    return ex;
}

template <class Item, class Get>
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(int64_t m, Get get, Item* tile_sums) {
    __shared__ Item sm[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanIpt;
    Item acc{};
#pragma unroll
    for (int k = 0; k < kScanIpt; ++k) {
        if (base + k < m) acc = acc + get(base + k);
    }
    Item total;
    block_exclusive_scan(acc, sm, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the tile totals in place; grand total to *total_out.
template <class Item>
__global__ void __launch_bounds__(kScanThreads) scan_tile_sums_kernel(Item* tile_sums, int64_t ntiles, Item* total_out) {
    __shared__ Item sm[kScanThreads];
    const int64_t per = (ntiles + kScanThreads - 1) / kScanThreads;
    const int64_t lo = (int64_t)threadIdx.x * per;
    const int64_t hi = min(ntiles, lo + per);
    Item acc{};
    for (int64_t k = lo; k < hi; ++k) acc = acc + tile_sums[k];
    Item total;
    Item run = block_exclusive_scan(acc, sm, total);
    for (int64_t k = lo; k < hi; ++k) {
        const Item v = tile_sums[k];
        tile_sums[k] = run;
        run = run + v;
    }
    if (threadIdx.x == 0) *total_out = total;
}

template <class Item, class Get, class Put>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(int64_t m, Get get, Put put, const Item* tile_offsets) {
    __shared__ Item sm[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanIpt;
    Item own[kScanIpt];
    Item acc{};
#pragma unroll
    for (int k = 0; k < kScanIpt; ++k) {
        own[k] = (base + k < m) ? get(base + k) : Item{};
        acc = acc + own[k];
    }
    Item total;
    Item run = block_exclusive_scan(acc, sm, total);
    run = tile_offsets[blockIdx.x] + run;
#pragma unroll
    for (int k = 0; k < kScanIpt; ++k) {
        if (base + k < m) put(base + k, run, own[k]);
        run = run + own[k];
    }
}

__global__ void store_totals_kernel(SetupWs ws, const ItemK* ktot, const ItemC* ctot) {
    if (ktot) {
        ws.info->T = ktot->k;
        if (ktot->k == 0 && ws.info->status == 0) ws.info->status = RK_EINVAL;
    }
    if (ctot) {
        ws.info->nl = ctot->nl;
        ws.info->nh = ctot->nh;
    }
}

// ---------------------------------------------------------------------------
// Alias table from the prefix sums (the parallel form of the sweep):
//  light at position k (exclusive deficit D_k): alias = heavy p with the
//    smallest inclusive excess E_p >= D_k; thr = S_i;
//  heavy at position p < nh-1: k* = first light with inclusive deficit > E_p;
//    thr = T + E_p - Dinc_{k*}, alias = heavy p+1;  the last heavy: thr = T, self;
//  S_i = T: thr = T, self.
// thr64 = floor(thr 2^64 / T), or UINT64_MAX when thr = T.
// ---------------------------------------------------------------------------
__global__ void alias_kernel(int64_t m, SetupWs ws) {
    if (ws.info->status != 0) return;
    const uint64_t T = ws.info->T;
    const uint32_t nl = ws.info->nl, nh = ws.info->nh;
    const u128 TT = (u128)T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const u128 S = (u128)(uint64_t)m * (u128)ws.K[i];
        u128 thr;
        uint32_t al;
        if (S < TT) {
            if (nh == 0) {  // impossible for a valid law; never index an empty list
                atomicCAS(&ws.info->status, 0, RK_EINVAL);
                continue;
            }
            const u128 D = ws.row_Dex[i];
            uint32_t lo = 0, hi = nh;  // first p with heavy_Einc[p] >= D
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (ws.heavy_Einc[mid] >= D) hi = mid; else lo = mid + 1;
            }
            if (lo >= nh) { atomicCAS(&ws.info->status, 0, RK_EINVAL); lo = nh - 1; }
            thr = S;
            al = ws.heavy_idx[lo];
        } else if (S > TT) {
            const uint32_t p = ws.row_pos[i];
            if (p + 1 == nh) {
                thr = TT;
                al = (uint32_t)i;
            } else if (nl == 0 || p >= nh) {  // impossible for a valid law
                atomicCAS(&ws.info->status, 0, RK_EINVAL);
                continue;
            } else {
                const u128 E = ws.heavy_Einc[p];
                uint32_t lo = 0, hi = nl;  // first k with light_Dinc[k] > E
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (ws.light_Dinc[mid] > E) hi = mid; else lo = mid + 1;
                }
                if (lo >= nl) { atomicCAS(&ws.info->status, 0, RK_EINVAL); lo = nl - 1; }
                thr = TT + E - ws.light_Dinc[lo];
                al = ws.heavy_idx[p + 1];
            }
        } else {
            thr = TT;
            al = (uint32_t)i;
        }
        ws.thr64[i] = (thr >= TT) ? ~0ull : (uint64_t)((thr << 64) / TT);
        ws.alias[i] = al;
    }
}

static int grid_for(int64_t m, int threads) {
    int64_t g = (m + threads - 1) / threads;
    if (g > 65535LL * 8) g = 65535LL * 8;
    return (int)(g < 1 ? 1 : g);
}

template <class LD, int NT, int S>
static void launch_row_weight_staged(const uint8_t* A, const float* row_scale, int64_t m, int64_t n,
                                     int64_t lda_bytes, const SetupWs& ws, int sms, cudaStream_t st) {
    const int64_t nchunks = (n + LD::kPerChunk - 1) / LD::kPerChunk;
    const size_t smem = (size_t)S * (size_t)nchunks * 16;
    auto kern = row_weight_staged_kernel<LD, NT, S>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    const int g = (int)std::min<int64_t>(m, (int64_t)sms * (per_sm < 1 ? 1 : per_sm));
    kern<<<g, NT, smem, st>>>(A, row_scale, m, n, lda_bytes, ws);
}

// Rows of more than 8 KB and up to 64 KB go to the staged CTA-per-row kernel
// (read once through a ring of cp.async stages, up to 128 KB a CTA); shorter
// rows (a warp a row re-reads them from L2 and needs no CTA barrier) and longer
// ones to the warp-per-row kernel.
template <class LD>
static void launch_row_weights(const uint8_t* A, const float* row_scale, int64_t m, int64_t n,
                               int64_t lda_bytes, const SetupWs& ws, int sms, cudaStream_t st) {
    const int64_t nchunks = (n + LD::kPerChunk - 1) / LD::kPerChunk;
    const int64_t row_bytes = nchunks * 16;
    if (row_bytes > 8 * 1024 && row_bytes <= 64 * 1024) {
        if (row_bytes <= 12 * 1024) launch_row_weight_staged<LD, 256, 8>(A, row_scale, m, n, lda_bytes, ws, sms, st);
        else if (row_bytes <= 24 * 1024) launch_row_weight_staged<LD, 256, 4>(A, row_scale, m, n, lda_bytes, ws, sms, st);
        else launch_row_weight_staged<LD, 256, 2>(A, row_scale, m, n, lda_bytes, ws, sms, st);
        return;
    }
    const int gw = (int)std::min<int64_t>((m + 7) / 8, (int64_t)sms * 8);   // 8 rows (warps) a CTA
    row_weight_kernel<LD><<<gw, 256, 0, st>>>(A, row_scale, m, n, lda_bytes, ws);
}

__global__ void setup_info_init_kernel(SetupInfo* info) {
    SetupInfo init{};
    init.H = kNoRows;
    *info = init;
}

int launch_setup(const void* A, rk_dtype dt, const float* row_scale, int64_t m, int64_t n,
                 int64_t lda, const SetupWs& ws, cudaStream_t st) {
    // the header is reset on the device (no host copy: the call stays capturable)
    setup_info_init_kernel<<<1, 1, 0, st>>>(ws.info);
    count_launch();
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint8_t* Ab = static_cast<const uint8_t*>(A);
    switch (dt) {
        case RK_F32:
            launch_row_weights<LoadF32>(Ab, nullptr, m, n, lda * 4, ws, sms, st);
            break;
        case RK_BF16:
            launch_row_weights<LoadBF16>(Ab, nullptr, m, n, lda * 2, ws, sms, st);
            break;
        case RK_FP8E4M3:
            launch_row_weights<LoadFP8>(Ab, row_scale, m, n, lda, ws, sms, st);
            break;
    }
    count_launch();
    weights_to_k_kernel<<<grid_for(m, 256), 256, 0, st>>>(m, ws);
    count_launch();
    const int64_t ntiles = (m + kScanTile - 1) / kScanTile;
    ItemK* ktiles = reinterpret_cast<ItemK*>(ws.tiles);
    ItemK* ktot = reinterpret_cast<ItemK*>(ws.tile_total);
    scan_tiles_kernel<ItemK, GetK><<<(unsigned)ntiles, kScanThreads, 0, st>>>(m, GetK{ws.K}, ktiles);
    scan_tile_sums_kernel<ItemK><<<1, kScanThreads, 0, st>>>(ktiles, ntiles, ktot);
    scan_apply_kernel<ItemK, GetK, PutK><<<(unsigned)ntiles, kScanThreads, 0, st>>>(m, GetK{ws.K}, PutK{ws.P}, ktiles);
    store_totals_kernel<<<1, 1, 0, st>>>(ws, ktot, nullptr);
    count_launch(4);
    ItemC* ctiles = reinterpret_cast<ItemC*>(ws.tiles);
    ItemC* ctot = reinterpret_cast<ItemC*>(ws.tile_total);
    GetC getc{ws.K, (uint64_t)m, ws.info};
    scan_tiles_kernel<ItemC, GetC><<<(unsigned)ntiles, kScanThreads, 0, st>>>(m, getc, ctiles);
    scan_tile_sums_kernel<ItemC><<<1, kScanThreads, 0, st>>>(ctiles, ntiles, ctot);
    scan_apply_kernel<ItemC, GetC, PutC><<<(unsigned)ntiles, kScanThreads, 0, st>>>(m, getc, PutC{ws}, ctiles);
    store_totals_kernel<<<1, 1, 0, st>>>(ws, nullptr, ctot);
    alias_kernel<<<grid_for(m, 256), 256, 0, st>>>(m, ws);
    count_launch(5);
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

size_t scan_tiles_bytes(int64_t m) {
    const int64_t ntiles = (m + kScanTile - 1) / kScanTile;
    return (size_t)ntiles * sizeof(ItemC);
}

size_t scan_item_bytes() { return sizeof(ItemC); }

}  // namespace rk
