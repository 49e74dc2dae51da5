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
    uint32_t* bloom = nullptr;        // blocked Bloom filter over the keys (NULL: none)
    uint64_t bloom_blocks = 0;        // 32-byte blocks, a power of two
};

namespace olap {

constexpr uint64_t JN_EMPTY = ~0ull;
constexpr int JB_TPB = 256;
constexpr int JP_TPB = 256;
constexpr int JP_STAGE = 6144;    // pairs staged per CTA (48 KB), split evenly over its warps
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

// Streaming probe-side traffic (keys, row-ids, pairs) is read or written
// once: the .cs forms allocate its L2 lines evict-first, so the table's lines
// are what L2 keeps.
__device__ __forceinline__ uint64_t ld_stream_u64(const void* p) {
    uint64_t v;
    asm volatile("ld.global.cs.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const void* p) {
    uint32_t v;
    asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream_pair(uint2* p, uint2 v) {
    asm volatile("st.global.cs.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(v.x), "r"(v.y) : "memory");
}

// Blocked Bloom filter (Putze, Sanders & Singler, "Cache-, hash- and
// space-efficient Bloom filters", WEA 2007): every key maps to one 32-byte
// block (one sector, one load) and sets one bit in each of the block's eight
// 32-bit words.  The block comes from bits 40..63 of fmix64(key), which the
// table's bucket index (the low bits) does not use; the eight bit positions
// come from 40 bits of a second hash, fmix64 of the complemented key.
constexpr int BLOOM_WORDS = 8;

__device__ __forceinline__ uint64_t bloom_block(uint64_t key, uint64_t bmask) {
    return (fmix64(key) >> 40) & bmask;
}
__device__ __forceinline__ uint32_t bloom_bit(uint64_t g, int w) {
    return 1u << static_cast<uint32_t>((g >> (5 * w)) & 31u);
}
// Whether `key` may be among the filter's keys (no false negatives).
__device__ __forceinline__ bool bloom_maybe(const uint32_t* bloom, uint64_t bmask, uint64_t key) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(bloom + bloom_block(key, bmask) * BLOOM_WORDS);
    uint64_t a, b, c, d;
    asm("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
    const uint64_t g = fmix64(~key);
    const uint64_t want01 = static_cast<uint64_t>(bloom_bit(g, 0)) | (static_cast<uint64_t>(bloom_bit(g, 1)) << 32);
    const uint64_t want23 = static_cast<uint64_t>(bloom_bit(g, 2)) | (static_cast<uint64_t>(bloom_bit(g, 3)) << 32);
    const uint64_t want45 = static_cast<uint64_t>(bloom_bit(g, 4)) | (static_cast<uint64_t>(bloom_bit(g, 5)) << 32);
    const uint64_t want67 = static_cast<uint64_t>(bloom_bit(g, 6)) | (static_cast<uint64_t>(bloom_bit(g, 7)) << 32);
    return (a & want01) == want01 && (b & want23) == want23 && (c & want45) == want45 && (d & want67) == want67;
}

// Device-side plan of one probe, written by its sampling stage: whether the
// Bloom pre-probe filters the rows (and how many it kept), and whether the
// probe skips the partition passes and reads its rows directly.  The stages
// after the sample read it, so the decision never travels through the host.
struct ProbeCtl {
    int active;                    // the pre-probe drops rows
    int direct;                    // the partition passes are skipped
    unsigned long long count;      // rows the pre-probe kept
    const int64_t* keys;           // with `redirect`: the rows the probe kernel reads
    const uint32_t* rowids;
    int redirect;
    int l1;                        // the probe's bucket reads go through L1
};

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

// One 32-byte bucket {key0, row-id0 | pad, key1, row-id1 | pad} in a single
// 256-bit load; L2_ONLY bypasses L1 (ld.global.cg), else the read-only path
// through L1 (ld.global.nc).
struct Bucket {
    uint64_t k0, w0, k1, w1;          // w: row-id in the low 32 bits, further copies in the high 32
};

template <bool L2_ONLY>
__device__ __forceinline__ Bucket ld_bucket(const ulonglong2* slots, uint32_t b) {
    const ulonglong2* p = slots + static_cast<uint64_t>(b) * 2;
    Bucket v;
    if (L2_ONLY)
        asm("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(v.k0), "=l"(v.w0), "=l"(v.k1), "=l"(v.w1) : "l"(p));
    else
        asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(v.k0), "=l"(v.w0), "=l"(v.k1), "=l"(v.w1) : "l"(p));
    return v;
}

constexpr int JP_S = 2;                                 // independent probe streams per lane
constexpr int JP_WARPS = JP_TPB / 32;
constexpr unsigned JP_WCAP = JP_STAGE / JP_WARPS;         // staged pairs per warp

// Copy a warp's staged pairs to the output with one atomic on the global
// count (whole warp calls; cnt is warp-uniform).
__device__ __forceinline__ void warp_flush(const ProbeArgs& a, uint2* ws, unsigned& cnt) {
    if (cnt == 0) return;
    __syncwarp();
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(a.count, static_cast<unsigned long long>(cnt));
    g = __shfl_sync(0xFFFFFFFFu, g, 0);
    for (unsigned i = lane; i < cnt; i += 32)
        if (g + i < a.cap) st_stream_pair(a.out + g + i, ws[i]);
    __syncwarp();
    cnt = 0;
}

// Stage one pair for every lane where m is set (whole warp calls).
__device__ __forceinline__ void warp_put(const ProbeArgs& a, uint2* ws, unsigned& cnt, bool m, uint2 p) {
    const unsigned b = __ballot_sync(0xFFFFFFFFu, m);
    if (b == 0) return;
    if (cnt + 32 > JP_WCAP) warp_flush(a, ws, cnt);
    const unsigned lane = threadIdx.x & 31u;
    if (m) ws[cnt + __popc(b & ((1u << lane) - 1u))] = p;
    cnt += __popc(b);
}

// Rows handed to the lanes of one warp.  The warp takes chunks of JQ_CHUNK
// consecutive rows from a global counter and gives them out in order, the
// lanes that need a row in one step getting consecutive rows, so the loads of
// their keys and row-ids coalesce.  Every field is warp-uniform: `cur` is the
// chunk being handed out, `nxt` the one taken after it (empty: b == e).
constexpr uint64_t JQ_CHUNK = 512;

struct RowRange {
    uint64_t b, e;
};

struct RowQueue {
    RowRange cur, nxt;
    unsigned long long* counter;  // next unclaimed row (zeroed before the launch)
    uint64_t n;
};

__device__ __forceinline__ RowRange take_chunk(RowQueue& q) {
    unsigned long long g = 0;
    if ((threadIdx.x & 31u) == 0) g = atomicAdd(q.counter, static_cast<unsigned long long>(JQ_CHUNK));
    g = __shfl_sync(0xFFFFFFFFu, g, 0);
    return RowRange{min(static_cast<uint64_t>(g), q.n), min(static_cast<uint64_t>(g) + JQ_CHUNK, q.n)};
}

// The next row of every lane in `need` (a ballot; whole warp calls): row
// index, or false when the rows are exhausted.
__device__ __forceinline__ bool queue_next(RowQueue& q, unsigned need, uint64_t* row) {
    const unsigned c = __popc(need);
    if (c == 0) return false;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned r = __popc(need & ((1u << lane) - 1u));
    uint64_t avail = q.cur.e - q.cur.b;
    if (avail < c && q.nxt.b == q.nxt.e) q.nxt = take_chunk(q);
    bool ok;
    if (r < avail) {
        *row = q.cur.b + r;
        ok = true;
    } else {
        *row = q.nxt.b + (r - avail);
        ok = *row < q.nxt.e;
    }
    if (c <= avail) {
        q.cur.b += c;
    } else {
        const uint64_t used = min(static_cast<uint64_t>(c) - avail, q.nxt.e - q.nxt.b);
        q.cur = RowRange{q.nxt.b + used, q.nxt.e};
        q.nxt = RowRange{0, 0};
    }
    return ok && ((need >> lane) & 1u);
}

// One warp probes rows from the queue until the rows run out.  Each lane runs
// JP_S independent streams.  A stream walks its row's chain one bucket per
// step and, when the chain ends, switches at once to the row it has already
// loaded and asks the queue for the next one.  Matches go to the warp's own
// stage `ws`, flushed to the output whenever it could overflow and at the end.
template <bool L2_ONLY, int S>
__device__ __forceinline__ void probe_queue(const ProbeArgs& a, RowQueue& q, uint2* ws) {
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t mask = static_cast<uint32_t>(a.mask);
    unsigned cnt = 0;
    uint64_t key[S], pkey[S];
    uint32_t rid[S], prid[S], bk[S];
    bool live[S], plive[S];
    Bucket v[S];
    q.cur = take_chunk(q);
    q.nxt = RowRange{0, 0};
    // current rows, then the rows loaded ahead
#pragma unroll
    for (int s = 0; s < S; ++s) {
        uint64_t i = 0;
        live[s] = queue_next(q, 0xFFFFFFFFu, &i);
        key[s] = live[s] ? ld_stream_u64(a.keys + i) : JN_EMPTY;
        rid[s] = live[s] ? (a.rowids ? ld_stream_u32(a.rowids + i) : static_cast<uint32_t>(i)) : 0u;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        uint64_t i = 0;
        plive[s] = queue_next(q, 0xFFFFFFFFu, &i);
        pkey[s] = plive[s] ? ld_stream_u64(a.keys + i) : JN_EMPTY;
        prid[s] = plive[s] ? (a.rowids ? ld_stream_u32(a.rowids + i) : static_cast<uint32_t>(i)) : 0u;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        bk[s] = static_cast<uint32_t>(fmix64(key[s])) & mask;
        v[s] = (live[s] && key[s] != JN_EMPTY) ? ld_bucket<L2_ONLY>(a.slots, bk[s]) : Bucket{JN_EMPTY, 0, JN_EMPTY, 0};
    }
    while (true) {
        bool any = false;
#pragma unroll
        for (int s = 0; s < S; ++s) any = any || live[s];
        if (!__any_sync(0xFFFFFFFFu, any)) break;
        // Probe keys equal to the empty marker pair with every side-list row;
        // the warp emits them together, one such key at a time (rare).  With
        // no side list such rows match nothing and are simply passed over.
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (a.n_side == 0) break;
            unsigned sb = __ballot_sync(0xFFFFFFFFu, live[s] && key[s] == JN_EMPTY);
            while (sb) {
                const int src = __ffs(sb) - 1;
                sb &= sb - 1;
                const uint32_t r = __shfl_sync(0xFFFFFFFFu, rid[s], src);
                for (uint64_t o0 = 0; o0 < a.n_side; o0 += 32) {
                    const bool m = o0 + lane < a.n_side;
                    warp_put(a, ws, cnt, m, make_uint2(r, m ? a.side[o0 + lane] : 0u));
                }
            }
        }
        // Matches in the current bucket of every stream; a match whose slot
        // counts no further copies of its key ends the row's walk.
        bool go[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const bool real = live[s] && key[s] != JN_EMPTY;
            const bool m0 = real && v[s].k0 == key[s], m1 = real && v[s].k1 == key[s];
            warp_put(a, ws, cnt, m0, make_uint2(rid[s], static_cast<uint32_t>(v[s].w0)));
            warp_put(a, ws, cnt, m1, make_uint2(rid[s], static_cast<uint32_t>(v[s].w1)));
            const bool last = (m0 && (v[s].w0 >> 32) == 0) || (m1 && (v[s].w1 >> 32) == 0);
            go[s] = real && !last && v[s].k1 != JN_EMPTY;     // slot 1 taken: the bucket is full
        }
        // Each stream steps along its chain, or takes the row it loaded ahead
        // and loads the queue's next row in its place.
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const bool swap = live[s] && !go[s];
            uint64_t i = 0;
            const bool got = queue_next(q, __ballot_sync(0xFFFFFFFFu, swap && plive[s]), &i);
            if (go[s]) {
                bk[s] = (bk[s] + 1u) & mask;
            } else if (swap) {
                live[s] = plive[s];
                key[s] = pkey[s];
                rid[s] = prid[s];
                bk[s] = static_cast<uint32_t>(fmix64(key[s])) & mask;
                plive[s] = got;
                if (got) {
                    pkey[s] = ld_stream_u64(a.keys + i);
                    prid[s] = a.rowids ? ld_stream_u32(a.rowids + i) : static_cast<uint32_t>(i);
                }
            }
            if (live[s] && key[s] != JN_EMPTY) v[s] = ld_bucket<L2_ONLY>(a.slots, bk[s]);
        }
    }
    warp_flush(a, ws, cnt);
}

}  // namespace olap
