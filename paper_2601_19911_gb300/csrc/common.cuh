// Shared device helpers of the GB300 OLAP library: order-preserving key
// transforms, (key, row-id) composite digits, warp-aggregated appends and a
// grid barrier whose wait is bounded.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "olap.h"

namespace olap {

constexpr uint64_t SIGN64 = 0x8000000000000000ull;

// Bound on any device-side wait: about one second at the GB300's clocks.
constexpr long long WAIT_LIMIT_CYCLES = 2000000000ll;

// ---------------------------------------------------------------------------
// Order-preserving transform of a key into an unsigned "rank word".  Selection
// in either order then becomes "smallest rank words first", with the row-id
// ascending as the second field of the composite (key, row-id) order.
//   signed integers: flip the sign bit (two's complement -> offset binary).
//   unsigned integers: the bits as they are.
//   floats: IEEE 754 totalOrder as an unsigned order: negative patterns are
//   inverted, non-negative ones get the sign bit set.
//   DESC: the word is complemented.
// A 4-byte key's word is left-aligned in 64 bits, so every rank word is 64
// bits and its first `key_bits` bits are significant.
// ---------------------------------------------------------------------------
// Every key type (olap_key_type): width and the rank word of raw key bits
// (4-byte keys in the low half of `bits`), and back.
__host__ __device__ __forceinline__ int key_bytes(int kind) {
    return (kind == OLAP_KEY_F32 || kind == OLAP_KEY_I32 || kind == OLAP_KEY_U32) ? 4 : 8;
}
__host__ __device__ __forceinline__ uint64_t rank_key(uint64_t bits, int kind, bool desc) {
    if (key_bytes(kind) == 8) {
        uint64_t u;
        if (kind == OLAP_KEY_I64) u = bits ^ SIGN64;
        else if (kind == OLAP_KEY_U64) u = bits;
        else u = (bits & SIGN64) ? ~bits : (bits | SIGN64);        // float64
        return desc ? ~u : u;
    }
    const uint32_t b = static_cast<uint32_t>(bits);
    uint32_t u;
    if (kind == OLAP_KEY_I32) u = b ^ 0x80000000u;
    else if (kind == OLAP_KEY_U32) u = b;
    else u = (b & 0x80000000u) ? ~b : (b | 0x80000000u);            // float32
    if (desc) u = ~u;
    return static_cast<uint64_t>(u) << 32;
}
__host__ __device__ __forceinline__ uint64_t unrank_key(uint64_t r, int kind, bool desc) {
    if (key_bytes(kind) == 8) {
        const uint64_t u = desc ? ~r : r;
        if (kind == OLAP_KEY_I64) return u ^ SIGN64;
        if (kind == OLAP_KEY_U64) return u;
        return (u & SIGN64) ? (u & ~SIGN64) : ~u;                   // float64
    }
    uint32_t u = static_cast<uint32_t>(r >> 32);
    if (desc) u = ~u;
    if (kind == OLAP_KEY_I32) return u ^ 0x80000000u;
    if (kind == OLAP_KEY_U32) return u;
    return (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : static_cast<uint32_t>(~u);
}

// ---------------------------------------------------------------------------
// Composite (rank word, row-id) as a 128-bit big-endian bit string (w0, w1):
// the key_bits significant bits of the rank word followed by the 32 row-id
// bits.  Total significant bits: key_bits + 32 (96 for int64, 64 for float32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void comp_words(uint64_t r, uint32_t rid, int key_bits, uint64_t& w0,
                                           uint64_t& w1) {
    if (key_bits == 64) {
        w0 = r;
        w1 = static_cast<uint64_t>(rid) << 32;
    } else {
        w0 = r | rid;
        w1 = 0;
    }
}

// Bits [L, L + d) of (w0, w1), MSB first; 1 <= d <= 32, L + d <= 128.
__device__ __forceinline__ uint32_t comp_digit(uint64_t w0, uint64_t w1, int L, int d) {
    uint64_t hi;
    if (L == 0)
        hi = w0;
    else if (L < 64)
        hi = (w0 << L) | (w1 >> (64 - L));
    else
        hi = w1 << (L - 64);
    return static_cast<uint32_t>(hi >> (64 - d));
}

// Compare the first L bits of (w0, w1) with the prefix (p0, p1): -1, 0, +1.
__device__ __forceinline__ int prefix_cmp(uint64_t w0, uint64_t w1, uint64_t p0, uint64_t p1, int L) {
    if (L == 0) return 0;
    if (L < 64) {
        const uint64_t m = ~0ull << (64 - L);
        const uint64_t a = w0 & m, b = p0 & m;
        return a < b ? -1 : (a > b ? 1 : 0);
    }
    if (w0 != p0) return w0 < p0 ? -1 : 1;
    if (L == 64) return 0;
    const uint64_t m = ~0ull << (128 - L);
    const uint64_t a = w1 & m, b = p1 & m;
    return a < b ? -1 : (a > b ? 1 : 0);
}

// Fold (w0, w1) into running AND / OR words.
__device__ __forceinline__ void and_or(uint64_t w0, uint64_t w1, uint64_t* ao) {
    ao[0] &= w0;
    ao[1] &= w1;
    ao[2] |= w0;
    ao[3] |= w1;
}

// Reduce the running AND / OR words over the CTA (warp shuffles, then the
// warps' results in shared memory) and merge them into `dst` with four
// atomics per CTA: same-address atomics serialise in L2, so one per warp
// would cost thousands of serial updates over the grid.  Whole CTA calls.
template <int TPB>
__device__ __forceinline__ void and_or_merge(uint64_t* ao, unsigned long long* dst) {
    __shared__ unsigned long long s_ao[TPB / 32][4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ao[0] &= __shfl_xor_sync(0xFFFFFFFFu, ao[0], o);
        ao[1] &= __shfl_xor_sync(0xFFFFFFFFu, ao[1], o);
        ao[2] |= __shfl_xor_sync(0xFFFFFFFFu, ao[2], o);
        ao[3] |= __shfl_xor_sync(0xFFFFFFFFu, ao[3], o);
    }
    if ((threadIdx.x & 31u) == 0)
        for (int j = 0; j < 4; ++j) s_ao[threadIdx.x >> 5][j] = ao[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t r[4] = {~0ull, ~0ull, 0ull, 0ull};
        for (int w = 0; w < TPB / 32; ++w) {
            r[0] &= s_ao[w][0];
            r[1] &= s_ao[w][1];
            r[2] |= s_ao[w][2];
            r[3] |= s_ao[w][3];
        }
        atomicAnd(dst + 0, static_cast<unsigned long long>(r[0]));
        atomicAnd(dst + 1, static_cast<unsigned long long>(r[1]));
        atomicOr(dst + 2, static_cast<unsigned long long>(r[2]));
        atomicOr(dst + 3, static_cast<unsigned long long>(r[3]));
    }
    __syncthreads();
}

// First bit position (0 = MSB of w0) where the entries behind merged AND / OR
// words differ; `total` when they agree everywhere.
__device__ __forceinline__ int first_diff(const unsigned long long* ao, int total) {
    const uint64_t d0 = __ldcg(ao + 0) ^ __ldcg(ao + 2), d1 = __ldcg(ao + 1) ^ __ldcg(ao + 3);
    const int f = d0 ? __clzll(static_cast<long long>(d0)) : (d1 ? 64 + __clzll(static_cast<long long>(d1)) : 128);
    return f < total ? f : total;
}

// Bits [lo, hi) of a 64-bit word counted from its MSB (0 <= lo <= hi <= 64).
__device__ __forceinline__ uint64_t bit_range(int lo, int hi) {
    if (hi <= lo) return 0ull;
    const uint64_t ones = (hi - lo == 64) ? ~0ull : ((1ull << (hi - lo)) - 1ull);
    return ones << (64 - hi);
}

// Copy bits [from, to) of (a0, a1) into (p0, p1), whose bits there are zero.
__device__ __forceinline__ void prefix_copy(uint64_t& p0, uint64_t& p1, uint64_t a0, uint64_t a1, int from, int to) {
    if (from < 64) p0 |= a0 & bit_range(from, to < 64 ? to : 64);
    if (to > 64) p1 |= a1 & bit_range((from > 64 ? from : 64) - 64, to - 64);
}

// Set bits [L, L + d) of (p0, p1) to `digit`.
__device__ __forceinline__ void prefix_set(uint64_t& p0, uint64_t& p1, int L, int d, uint32_t digit) {
    const uint64_t v = static_cast<uint64_t>(digit);
    if (L + d <= 64) {
        p0 |= v << (64 - L - d);
    } else if (L >= 64) {
        p1 |= v << (128 - L - d);
    } else {                                  // straddles the word boundary
        const int in0 = 64 - L;               // bits of the digit that land in p0
        p0 |= v >> (d - in0);
        p1 |= v << (64 - (d - in0));
    }
}

// ---------------------------------------------------------------------------
// Memory-order helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

// Grid barrier for cooperative launches (all CTAs co-resident).  Arrival is an
// atomic count; the last CTA to arrive resets it and bumps a generation word
// the others wait on.  The wait is bounded: after WAIT_LIMIT_CYCLES the CTA
// records OLAP_E_TIMEOUT in *err and leaves; callers test the return value
// and stop.  The counter returns to zero after every completed barrier.
struct GridBar {
    unsigned count;
    unsigned gen;
    unsigned prep;        // tickets of the Top-K prepare kernel's CTAs (a multiple of its grid between launches)
    unsigned pad;
};

// Wait until *word differs from `old`, at most `limit` clock cycles; on
// expiry record OLAP_E_TIMEOUT in *err (first error wins) and return false.
__device__ __forceinline__ bool wait_changed(const unsigned* word, unsigned old, int* err, long long limit) {
    const long long t0 = clock64();
    while (ld_acquire_u32(word) == old) {
        if (clock64() - t0 > limit) {
            atomicCAS(err, 0, static_cast<int>(OLAP_E_TIMEOUT));
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ bool grid_sync(GridBar* bar, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
        const unsigned g = ld_acquire_u32(&bar->gen);
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            st_release_u32(&bar->gen, g + 1);
        } else {
            wait_changed(&bar->gen, g, err, WAIT_LIMIT_CYCLES);
        }
        __threadfence();
    }
    __syncthreads();
    return ld_volatile_i32(err) == 0;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine, non-tensor form) into shared memory,
// completed through an mbarrier transaction count.  Waits are bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, signalling `bar` on completion.
// The L2 policy marks the streamed lines evict-first.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                        uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Wait until phase `parity` of `bar` completes; false if the bound expires.
// Each try suspends the thread (hint: up to 10 ms) until the phase completes,
// so waiting warps do not spin on the issue slots the working warps need.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(10000000u)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
    }
}
__device__ __forceinline__ uint4 ld_shared_v4(const void* p) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}

// Warp-aggregated append: every lane contributes `cnt` items; returns the
// lane's first slot in a global array advanced by one atomic per warp.
__device__ __forceinline__ unsigned long long warp_append(unsigned long long* counter, unsigned cnt) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= static_cast<unsigned>(o)) incl += v;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(counter, static_cast<unsigned long long>(total));
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + (incl - cnt);
}

}  // namespace olap
