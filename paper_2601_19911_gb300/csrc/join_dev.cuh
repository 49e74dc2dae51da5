// Device side of the key-only hash join shared by the probe kernel and the
// batched executor: table constants, the fmix64 hash, the per-CTA staged
// output and the probe rounds.
#pragma once

#include <cstdint>

#include "common.cuh"

struct olap_join_table {
    olap_ctx* owner = nullptr;        // context whose budget counts this table (or NULL)
    int device = 0;
    ulonglong2* slots = nullptr;      // n_buckets * 2 slots
    uint64_t n_buckets = 0;
    uint32_t* side = nullptr;         // row-ids of build rows with the empty-marker key
    uint64_t n_side = 0;
    uint64_t n_build = 0;
    double load = 0.0;
    size_t bytes = 0;
};

namespace olap {

constexpr uint64_t JN_EMPTY = ~0ull;
constexpr int JB_TPB = 256;
constexpr int JP_TPB = 256;
constexpr int JP_U = 4;
constexpr int JP_STAGE = 6144;    // pairs staged per CTA (48 KB)
constexpr int JP_FLUSH = 2048;    // flush once this many are staged; a round adds at most
                                  // JP_TPB * JP_U * 2 per chain step, and the stage spills
                                  // to direct global appends if a round overfills it
constexpr int JP_SMEM = JP_STAGE * 8;

struct JoinCtl {
    unsigned long long side_count;   // build rows with the empty-marker key
    unsigned long long side_fill;
    int err;
    int pad;
};

__device__ __forceinline__ uint64_t fmix64(uint64_t h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

__device__ __forceinline__ uint64_t ld_stream_u64(const void* p) {
    uint64_t v;
    asm volatile("ld.global.cs.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

struct ProbeArgs {
    const int64_t* keys;
    const uint32_t* rowids;
    uint64_t n;
    const ulonglong2* slots;
    uint64_t mask;
    const uint32_t* side;
    uint64_t n_side;
    uint2* out;
    uint64_t cap;
    unsigned long long* count;
};

// Place one pair at stage position pos, or append it to the output directly
// once the stage is full.
__device__ __forceinline__ void put_pair(const ProbeArgs& a, uint2* stage, unsigned pos, uint2 p) {
    if (pos < JP_STAGE) {
        stage[pos] = p;
    } else {
        const unsigned long long g = atomicAdd(a.count, 1ull);
        if (g < a.cap) a.out[g] = p;
    }
}

// Warp-aggregated append of up to two pairs per lane (all lanes call).
__device__ __forceinline__ void warp_emit2(const ProbeArgs& a, uint2* stage, unsigned* scount, bool m0, uint2 p0,
                                           bool m1, uint2 p1) {
    const unsigned b0 = __ballot_sync(0xFFFFFFFFu, m0);
    const unsigned b1 = __ballot_sync(0xFFFFFFFFu, m1);
    const unsigned tot = __popc(b0) + __popc(b1);
    if (tot == 0) return;
    const unsigned lane = threadIdx.x & 31u;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(scount, tot);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    const unsigned lt = (1u << lane) - 1u;
    if (m0) put_pair(a, stage, base + __popc(b0 & lt), p0);
    if (m1) put_pair(a, stage, base + __popc(b0) + __popc(b1 & lt), p1);
}

// Copy the staged pairs to the output (whole CTA; call between barriers).
__device__ __forceinline__ void flush_stage(const ProbeArgs& a, uint2* stage, unsigned* scount,
                                            unsigned long long* sbase) {
    const unsigned c = min(*reinterpret_cast<volatile unsigned*>(scount), static_cast<unsigned>(JP_STAGE));
    if (threadIdx.x == 0) *sbase = c ? atomicAdd(a.count, static_cast<unsigned long long>(c)) : 0ull;
    __syncthreads();
    const unsigned long long base = *sbase;
    for (unsigned i = threadIdx.x; i < c; i += JP_TPB) {
        const unsigned long long g = base + i;
        if (g < a.cap) a.out[g] = stage[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) *scount = 0;
    __syncthreads();
}

// Probe rounds first, first + step, ... of JP_TPB * JP_U keys each by one CTA
// (whole CTA calls), over probe rows below `end` (at most a.n), staging pairs
// in `stage` (JP_STAGE entries) and flushing them to the output; everything
// staged is flushed before returning.
__device__ __forceinline__ void probe_rounds(const ProbeArgs& a, uint64_t first, uint64_t step, uint64_t end,
                                             uint2* stage, unsigned* scount_p, unsigned long long* sbase_p) {
    unsigned& scount = *scount_p;
    if (threadIdx.x == 0) scount = 0;
    __syncthreads();
    const uint64_t per = static_cast<uint64_t>(JP_TPB) * JP_U;
    for (uint64_t base = first * per; base < end; base += step * per) {
        uint64_t k[JP_U], bk[JP_U];
        uint32_t prid[JP_U];
        bool act[JP_U];
        ulonglong2 x0[JP_U], x1[JP_U];
#pragma unroll
        for (int j = 0; j < JP_U; ++j) {
            const uint64_t idx = base + static_cast<uint64_t>(j) * JP_TPB + threadIdx.x;
            const bool v = idx < end;
            k[j] = v ? ld_stream_u64(a.keys + idx) : JN_EMPTY;
            prid[j] = v ? (a.rowids ? a.rowids[idx] : static_cast<uint32_t>(idx)) : 0u;
            act[j] = v && k[j] != JN_EMPTY;
            // Probe keys equal to the empty marker pair with the side list.
            if (v && k[j] == JN_EMPTY)
                for (uint64_t o = 0; o < a.n_side; ++o)
                    put_pair(a, stage, atomicAdd(&scount, 1u), make_uint2(prid[j], a.side[o]));
        }
#pragma unroll
        for (int j = 0; j < JP_U; ++j) {
            bk[j] = act[j] ? (fmix64(k[j]) & a.mask) : 0;
            if (act[j]) {
                x0[j] = __ldg(a.slots + bk[j] * 2);
                x1[j] = __ldg(a.slots + bk[j] * 2 + 1);
            } else {
                x0[j] = make_ulonglong2(JN_EMPTY, 0);
                x1[j] = make_ulonglong2(JN_EMPTY, 0);
            }
        }
#pragma unroll
        for (int j = 0; j < JP_U; ++j) {
            bool on = act[j];
            while (__any_sync(0xFFFFFFFFu, on)) {
                const bool m0 = on && x0[j].x == k[j];
                const bool m1 = on && x1[j].x == k[j];
                warp_emit2(a, stage, &scount, m0, make_uint2(prid[j], static_cast<uint32_t>(x0[j].y)), m1,
                           make_uint2(prid[j], static_cast<uint32_t>(x1[j].y)));
                on = on && x0[j].x != JN_EMPTY && x1[j].x != JN_EMPTY;
                if (on) {
                    bk[j] = (bk[j] + 1) & a.mask;
                    x0[j] = __ldg(a.slots + bk[j] * 2);
                    x1[j] = __ldg(a.slots + bk[j] * 2 + 1);
                }
            }
        }
        __syncthreads();
        if (*reinterpret_cast<volatile unsigned*>(&scount) >= static_cast<unsigned>(JP_FLUSH))
            flush_stage(a, stage, &scount, sbase_p);
    }
    __syncthreads();
    flush_stage(a, stage, &scount, sbase_p);
}

}  // namespace olap
