// Block-level building blocks shared by the Top-K kernels (grid-wide and
// per-CTA): composite ordering, block scan, histogram bucket pick, shared
// memory bitonic sort, streaming loads and the key-domain threshold test.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace olap {

constexpr int PICK_BINS = 4096;   // histogram bins of a 12-bit digit

__device__ __forceinline__ bool elem_less(uint64_t ar, uint32_t arid, uint64_t br, uint32_t brid) {
    return ar < br || (ar == br && arid < brid);
}

__device__ __forceinline__ uint4 ld_stream_v4(const void* p) {
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Block-wide exclusive scan over one value per thread (TPB threads, <= 1024).
template <int TPB>
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* warp_sums,
                                                              unsigned long long* total) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= static_cast<unsigned>(o)) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = TPB / 32;
        unsigned long long w = lane < NW ? warp_sums[lane] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= static_cast<unsigned>(o)) wi += t;
        }
        if (lane < NW) warp_sums[lane] = wi - w;
        if (lane == NW - 1) *total = wi;
    }
    __syncthreads();
    const unsigned long long r = warp_sums[warp] + incl - v;
    __syncthreads();
    return r;
}

// Find the bucket b of a PICK_BINS histogram where the running count first
// reaches `need` (1 <= need <= total).  Every thread gets b, the count below b
// and the count in b.
struct Pick {
    unsigned b;
    unsigned long long below;
    unsigned long long in_b;
};

template <int TPB>
__device__ Pick pick_bucket(const unsigned* hist, unsigned long long need, unsigned long long* sc) {
    constexpr int PER = PICK_BINS / TPB;
    unsigned v[PER];
    unsigned long long local = 0;
    const volatile unsigned* h = hist;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        v[j] = h[threadIdx.x * PER + j];
        local += v[j];
    }
    unsigned long long* warp_sums = sc;        // 16 entries
    unsigned long long* total = sc + 16;
    unsigned long long* res = sc + 17;         // b, below, in_b
    const unsigned long long before = block_excl_scan<TPB>(local, warp_sums, total);
    if (before < need && need <= before + local) {
        unsigned long long run = before;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            if (run < need && need <= run + v[j]) {
                res[0] = threadIdx.x * PER + j;
                res[1] = run;
                res[2] = v[j];
            }
            run += v[j];
        }
    }
    __syncthreads();
    Pick p{static_cast<unsigned>(res[0]), res[1], res[2]};
    __syncthreads();
    return p;
}

// Bitonic sort of `count` entries in shared memory (room for the next power of two), ascending
// by (r, rid); padded to a power of two with all-ones entries.
template <int TPB>
__device__ void block_sort(uint64_t* sr, uint32_t* srid, int count) {
    int m = 1;
    while (m < count) m <<= 1;
    for (int i = count + threadIdx.x; i < m; i += TPB) {
        sr[i] = ~0ull;
        srid[i] = ~0u;
    }
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (m >> 1); t += TPB) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const uint64_t a = sr[lo], b = sr[hi];
                const uint32_t ar = srid[lo], br = srid[hi];
                const bool swap = up ? elem_less(b, br, a, ar) : elem_less(a, ar, b, br);
                if (swap) {
                    sr[lo] = b;
                    sr[hi] = a;
                    srid[lo] = br;
                    srid[hi] = ar;
                }
            }
            __syncthreads();
        }
    }
}

// The threshold of the streaming pass moved into the key domain, so that a
// key is tested with one XOR and one unsigned comparison and no transform:
// `rank <= t` holds exactly when `(key ^ m) >= c` for the (m, c) below (m64 /
// c64 for 8-byte keys, m32 / c32 for 4-byte keys, whose rank is t's upper
// half t32 = t >> 32; the lower half of a 4-byte key's rank is zero).
//   signed integers: rank = key ^ SIGN (ASC) or its complement (DESC); the
//     signed key order is the unsigned order of key ^ SIGN, and "<=" becomes
//     ">=" on the complement.
//   unsigned integers: ASC  key <= t  <=>  ~key >= ~t;  DESC  ~key <= t  <=>  key >= ~t.
//   floats: with y = x ^ ((x >> (w-1)) & MAG) the signed image of totalOrder
//     (MAG = all bits but the sign) and L the signed limit on y, each of the
//     four cases (order x sign of L) is one unsigned comparison of x under a
//     fixed XOR mask:
//       DESC, L >= 0: y >= L  <=>  x ^ SIGN >= L ^ SIGN
//       DESC, L <  0: y >= L  <=>  ~x >= ~(L ^ MAG)
//       ASC,  L >= 0: y <= L  <=>  x ^ MAG >= L ^ MAG
//       ASC,  L <  0: y <= L  <=>  x >= L ^ MAG
//     (XOR with MAG reverses the signed order among negative values.)
struct KeyLimit {
    uint64_t m64, c64;
    uint32_t m32, c32;
};

template <typename U>
__device__ __forceinline__ void float_limit(U t, bool desc, U* m, U* c) {
    constexpr U SIGN = static_cast<U>(1) << (sizeof(U) * 8 - 1);
    constexpr U MAG = ~SIGN;
    const U uL = (desc ? static_cast<U>(~t) : t) ^ SIGN;          // signed limit on y, as bits
    const bool neg = (uL & SIGN) != 0;
    if (desc) {
        if (!neg) { *m = SIGN; *c = uL ^ SIGN; }
        else      { *m = static_cast<U>(~static_cast<U>(0)); *c = static_cast<U>(~(uL ^ MAG)); }
    } else {
        if (!neg) { *m = MAG; *c = uL ^ MAG; }
        else      { *m = 0;   *c = uL ^ MAG; }
    }
}

template <typename U>
__device__ __forceinline__ void int_limit(U t, bool desc, bool is_signed, U* m, U* c) {
    constexpr U SIGN = static_cast<U>(1) << (sizeof(U) * 8 - 1);
    if (is_signed) {
        const U lim = (desc ? static_cast<U>(~t) : t) ^ SIGN;      // signed limit on the key
        *m = desc ? SIGN : static_cast<U>(~SIGN);
        *c = lim ^ *m;
    } else {
        *m = desc ? static_cast<U>(0) : static_cast<U>(~static_cast<U>(0));
        *c = static_cast<U>(~t);
    }
}

__device__ __forceinline__ KeyLimit key_limit(uint64_t t, int kind, bool desc) {
    KeyLimit k{0, 0, 0, 0};
    const uint32_t t32 = static_cast<uint32_t>(t >> 32);
    switch (kind) {
        case OLAP_KEY_I64: int_limit<uint64_t>(t, desc, true, &k.m64, &k.c64); break;
        case OLAP_KEY_U64: int_limit<uint64_t>(t, desc, false, &k.m64, &k.c64); break;
        case OLAP_KEY_F64: float_limit<uint64_t>(t, desc, &k.m64, &k.c64); break;
        case OLAP_KEY_I32: int_limit<uint32_t>(t32, desc, true, &k.m32, &k.c32); break;
        case OLAP_KEY_U32: int_limit<uint32_t>(t32, desc, false, &k.m32, &k.c32); break;
        default: float_limit<uint32_t>(t32, desc, &k.m32, &k.c32); break;   // float32
    }
    return k;
}
__device__ __forceinline__ bool pass64(uint64_t bits, const KeyLimit& k) { return (bits ^ k.m64) >= k.c64; }
__device__ __forceinline__ bool pass32(uint32_t bits, const KeyLimit& k) { return (bits ^ k.m32) >= k.c32; }

}  // namespace olap
