// Batched execution of many key-only Top-K queries and join probe batches in
// one persistent launch fed by a device work queue, captured in a CUDA graph.
//
// Small queries are where "kernel launching and transfer overheads are
// dominant" (Sec. IV, small-N interval).  Here one CTA runs one work item
// start to finish; CTAs take the next item from an atomic queue head, items
// sorted largest first on the host, so thousands of uneven items cost one
// launch.  A Top-K item larger than one CTA's share of the batch is split
// into parts that run as items of their own; a second launch merges each
// split item's parts.  Per item:
//   * Top-K (K <= 4096): a stratified sample of 2048 keys gives a threshold
//     rank word; one streaming pass appends the keys at or below it to the
//     CTA's own candidate buffer (no global atomics); block-local radix passes
//     over the candidates find the bucket of the K-th entry; the split puts
//     the selected entries in shared memory, where they are sorted.  Small
//     items (n <= 4096) are sorted whole; a misjudged sample falls back to
//     radix passes over the item's keys.
//   * probe: the probe loop of the join kernel over one chunk of at most
//     BP_CHUNK probe rows of an item, handed to the CTA's warps by a row
//     queue in shared memory; a large item is many chunks taken by many
//     CTAs, all appending to the item's own count word, which a reset kernel
//     zeroes before the probe queue starts.
// Descriptors are checked on the device; a bad one gets OLAP_E_DEVICE in its
// status word and is skipped.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "block.cuh"
#include "ctx.h"
#include "join_dev.cuh"

namespace olap {

namespace {

constexpr int BT_TPB = 512;
constexpr int BT_SMALL = 4096;            // entries one sort handles
constexpr int BT_SAMPLE = 2048;           // sample keys per item
constexpr int BT_SPT = BT_SAMPLE / BT_TPB;
constexpr uint32_t BT_CAND = 65536;       // candidate capacity per CTA
constexpr int BT_WS = 128;                // staged hits per warp
constexpr int BT_BINS = 4096;
constexpr int BT_SMEM = 2 * BT_SMALL * 12; // two sort areas; also the histogram, stages, probe stage
constexpr uint64_t BP_CHUNK = 32768;       // probe rows per work unit
constexpr uint64_t BT_SPLIT_N = 1ull << 19;  // smallest Top-K item that may be split into parts
constexpr uint64_t BT_PART = 1ull << 18;     // smallest target rows per part (parts are balanced)
static_assert(JP_STAGE * 8 <= BT_SMEM, "probe stage must fit");
static_assert((BT_TPB / 32) * BT_WS * 12 <= BT_SMEM, "warp stages must fit");

struct __align__(8) Item {
    int op;                      // OLAP_OP_TOPK / OLAP_OP_PROBE
    int w4;                      // 4-byte keys
    int desc;
    int kind;                    // olap_key_type
    const void* keys;
    const uint32_t* rowids;
    uint64_t n;
    uint64_t k;
    void* out_keys;
    uint32_t* out_rowids;
    const uint64_t* table;       // probe: buckets of 2 x 16-byte slots
    uint64_t mask;
    const uint32_t* side;
    uint64_t n_side;
    uint2* out_pairs;
    uint64_t cap;
    unsigned long long* count;   // rows (Top-K) or pairs (probe) written
    int32_t* status;
    uint64_t rowid_base;         // implicit row-ids: rowid_base + index
    int out_mode;                // Top-K output: ITEM_OUT_KEYS, ITEM_OUT_RANKS or ITEM_OUT_MERGE
    int out_kind;                // ITEM_OUT_MERGE: key kind and order of the original query
    int out_desc;
    int pad;
};

// How a Top-K item writes its result.  A large item is split into parts that
// each select their own Top-K and write rank words (ITEM_OUT_RANKS); a merge
// item then selects the Top-K of the parts' results (keys are rank words,
// read as uint64 ascending, with explicit row-ids) and writes the original
// key bits (ITEM_OUT_MERGE).
enum { ITEM_OUT_KEYS = 0, ITEM_OUT_RANKS = 1, ITEM_OUT_MERGE = 2 };

// One probe work unit: rows [chunk * BP_CHUNK, (chunk + 1) * BP_CHUNK) of probe
// item `item` (the last chunk of an item is shorter).
struct ProbeChunk {
    uint32_t item;
    uint32_t chunk;
};

__device__ __forceinline__ uint64_t item_rank(const Item& it, uint64_t i, uint32_t* rid) {
    uint64_t r;
    const uint64_t bits = it.w4 ? static_cast<uint64_t>(static_cast<const uint32_t*>(it.keys)[i])
                                : static_cast<const uint64_t*>(it.keys)[i];
    r = rank_key(bits, it.kind, it.desc);
    *rid = it.rowids ? it.rowids[i] : static_cast<uint32_t>(it.rowid_base + i);
    return r;
}

__device__ __forceinline__ void put_result(const Item& it, uint64_t i, uint64_t r, uint32_t rid) {
    if (it.out_mode == ITEM_OUT_RANKS) {
        static_cast<uint64_t*>(it.out_keys)[i] = r;
    } else if (it.out_mode == ITEM_OUT_MERGE) {
        // r is the rank word of the original key (uint64 ascending is identity)
        if (key_bytes(it.out_kind) == 4)
            static_cast<uint32_t*>(it.out_keys)[i] = static_cast<uint32_t>(unrank_key(r, it.out_kind, it.out_desc));
        else
            static_cast<uint64_t*>(it.out_keys)[i] = unrank_key(r, it.out_kind, it.out_desc);
    } else if (it.w4) {
        static_cast<uint32_t*>(it.out_keys)[i] = static_cast<uint32_t>(unrank_key(r, it.kind, it.desc));
    } else {
        static_cast<uint64_t*>(it.out_keys)[i] = unrank_key(r, it.kind, it.desc);
    }
    it.out_rowids[i] = rid;
}

// Threshold rank word from a stratified sample: radix select (digit bits) with the
// early exit of the grid version (between r and r + 8 samples at or below).
__device__ uint64_t cta_sample_threshold(const Item& it, unsigned r, unsigned* hist, unsigned long long* sc,
                                         int digit) {
    uint64_t s[BT_SPT];
#pragma unroll
    for (int j = 0; j < BT_SPT; ++j) {
        const uint64_t idx = static_cast<uint64_t>(j) * BT_TPB + threadIdx.x;
        const uint64_t pos = (idx * it.n) / BT_SAMPLE + (it.n / BT_SAMPLE) / 2;
        uint32_t rid;
        s[j] = item_rank(it, pos, &rid);
    }
    const int kb = it.w4 ? 32 : 64;
    uint64_t prefix = 0;
    unsigned long long rem = r, cum = 0;
    for (int L = 0; L < kb; L += digit) {
        const int d = min(digit, kb - L);
        for (int b = threadIdx.x; b < BT_BINS; b += BT_TPB) hist[b] = 0;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < BT_SPT; ++j) {
            const bool match = (L == 0) || (((s[j] ^ prefix) >> (64 - L)) == 0);
            if (match) atomicAdd(&hist[static_cast<unsigned>((s[j] << L) >> (64 - d))], 1u);
        }
        __syncthreads();
        const Pick pk = pick_bucket<BT_TPB>(hist, rem, sc);
        prefix |= static_cast<uint64_t>(pk.b) << (64 - L - d);
        rem -= pk.below;
        cum += pk.below;
        if (cum + pk.in_b <= r + 8) return prefix | ((1ull << (64 - L - d)) - 1ull);
    }
    return prefix;
}

// Move a warp's staged hits to the CTA's candidate buffer.
__device__ __forceinline__ void cta_flush_stage(uint64_t* ws_r, uint32_t* ws_idx, unsigned& cnt, const Item& it,
                                                uint64_t* cand_r, uint32_t* cand_rid, unsigned* s_cand) {
    if (cnt == 0) return;
    __syncwarp();
    const unsigned lane = threadIdx.x & 31u;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(s_cand, cnt);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (unsigned j = lane; j < cnt; j += 32) {
        if (base + j < BT_CAND) {
            const uint32_t idx = ws_idx[j];
            cand_r[base + j] = ws_r[j];
            cand_rid[base + j] = it.rowids ? it.rowids[idx] : static_cast<uint32_t>(it.rowid_base + idx);
        }
    }
    __syncwarp();
    cnt = 0;
}

// Test one key (rank via the key-domain limit) and stage a hit; the whole
// warp calls with its lanes' keys.
template <bool W4>
__device__ __forceinline__ void cta_filter_key(const Item& it, const KeyLimit& lim, bool valid, uint64_t bits,
                                               uint64_t idx, uint64_t* ws_r, uint32_t* ws_idx, unsigned& cnt,
                                               uint64_t* cand_r, uint32_t* cand_rid, unsigned* s_cand) {
    const bool hit = valid && (W4 ? pass32(static_cast<uint32_t>(bits), lim) : pass64(bits, lim));
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
    if (!bal) return;
    if (cnt + __popc(bal) > BT_WS) cta_flush_stage(ws_r, ws_idx, cnt, it, cand_r, cand_rid, s_cand);
    const unsigned lane = threadIdx.x & 31u;
    if (hit) {
        const unsigned pos = cnt + __popc(bal & ((1u << lane) - 1u));
        ws_r[pos] = rank_key(bits, it.kind, it.desc);
        ws_idx[pos] = static_cast<uint32_t>(idx);
    }
    cnt += __popc(bal);
}

// The streaming pass of one item by one CTA.  Returns the candidate count.
template <bool W4>
__device__ unsigned cta_filter(const Item& it, uint64_t t, unsigned char* smem, uint64_t* cand_r,
                               uint32_t* cand_rid, unsigned* s_cand) {
    const KeyLimit lim = key_limit(t, it.kind, it.desc);
    const unsigned w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    uint64_t* ws_r = reinterpret_cast<uint64_t*>(smem + w * BT_WS * 12);
    uint32_t* ws_idx = reinterpret_cast<uint32_t*>(smem + w * BT_WS * 12 + BT_WS * 8);
    unsigned cnt = 0;
    if (threadIdx.x == 0) *s_cand = 0;
    __syncthreads();
    constexpr int W = W4 ? 4 : 8;
    const uint64_t n = it.n;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(it.keys);
    const uint64_t head0 = ((16 - (addr & 15)) & 15) / W;
    const uint64_t head = head0 < n ? head0 : n;
    constexpr uint64_t VEC = 16 / W;
    const uint64_t nvec = (n - head) / VEC;
    const uint64_t tail0 = head + nvec * VEC;
    const unsigned char* vbase = static_cast<const unsigned char*>(it.keys) + head * W;
    // vectors: 4 in flight per thread
    for (uint64_t bb = 0; bb < nvec; bb += 4 * BT_TPB) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t vi = bb + static_cast<uint64_t>(u) * BT_TPB + threadIdx.x;
            v[u] = vi < nvec ? ld_stream_v4(vbase + vi * 16) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t vi = bb + static_cast<uint64_t>(u) * BT_TPB + threadIdx.x;
            const bool ok = vi < nvec;
            const uint64_t i0 = head + vi * VEC;
            if (W4) {
                const uint32_t x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    cta_filter_key<W4>(it, lim, ok, x[e], i0 + e, ws_r, ws_idx, cnt, cand_r, cand_rid, s_cand);
            } else {
                cta_filter_key<W4>(it, lim, ok, static_cast<uint64_t>(v[u].x) | (static_cast<uint64_t>(v[u].y) << 32),
                               i0, ws_r, ws_idx, cnt, cand_r, cand_rid, s_cand);
                cta_filter_key<W4>(it, lim, ok, static_cast<uint64_t>(v[u].z) | (static_cast<uint64_t>(v[u].w) << 32),
                               i0 + 1, ws_r, ws_idx, cnt, cand_r, cand_rid, s_cand);
            }
        }
    }
    // head and tail (at most 2 * VEC - 2 keys) by warp 0
    if (w == 0) {
        const uint64_t rest = head + (n - tail0);
        const bool ok = lane < rest;
        uint64_t idx = 0, bits = 0;
        if (ok) {
            idx = lane < head ? lane : tail0 + (lane - head);
            bits = W4 ? static_cast<const uint32_t*>(it.keys)[idx] : static_cast<const uint64_t*>(it.keys)[idx];
        }
        cta_filter_key<W4>(it, lim, ok, bits, idx, ws_r, ws_idx, cnt, cand_r, cand_rid, s_cand);
    }
    cta_flush_stage(ws_r, ws_idx, cnt, it, cand_r, cand_rid, s_cand);
    __syncthreads();
    return *reinterpret_cast<volatile unsigned*>(s_cand);
}

__device__ __forceinline__ void src_get(const Item& it, bool cand, const uint64_t* cand_r, const uint32_t* cand_rid,
                                        uint64_t i, uint64_t& r, uint32_t& rid) {
    if (cand) {
        r = cand_r[i];
        rid = cand_rid[i];
    } else {
        r = item_rank(it, i, &rid);
    }
}

// Top-K of one item by one CTA.
__device__ void cta_topk(const Item& it, unsigned char* smem, uint64_t* cand_r, uint32_t* cand_rid,
                         unsigned long long* sc, unsigned* s_misc, int digit) {
    const uint64_t n = it.n;
    const uint64_t kk = it.k < n ? it.k : n;
    if (kk == 0) {
        if (threadIdx.x == 0) *it.count = 0;
        return;
    }
    uint64_t* sr = reinterpret_cast<uint64_t*>(smem);
    uint32_t* srid = reinterpret_cast<uint32_t*>(smem + 2 * BT_SMALL * 8);
    unsigned* hist = reinterpret_cast<unsigned*>(smem);
    if (n <= BT_SMALL) {
        for (uint64_t i = threadIdx.x; i < n; i += BT_TPB) sr[i] = item_rank(it, i, &srid[i]);
        __syncthreads();
        block_sort<BT_TPB>(sr, srid, static_cast<int>(n));
        for (uint64_t i = threadIdx.x; i < kk; i += BT_TPB) put_result(it, i, sr[i], srid[i]);
        if (threadIdx.x == 0) *it.count = kk;
        return;
    }
    const int kb = it.w4 ? 32 : 64;
    const int TB = kb + 32;
    bool cand = false;
    uint64_t src_n = n;
    int L = 0;
    if (kk <= n / 16) {
        const double lam = static_cast<double>(kk) * BT_SAMPLE / static_cast<double>(n);
        unsigned r = static_cast<unsigned>(ceil(lam + 4.0 * sqrt(lam))) + 3u;
        if (r > BT_SAMPLE) r = BT_SAMPLE;
        const uint64_t t = cta_sample_threshold(it, r, hist, sc, digit);
        __syncthreads();
        const unsigned c = it.w4 ? cta_filter<true>(it, t, smem, cand_r, cand_rid, &s_misc[0])
                                  : cta_filter<false>(it, t, smem, cand_r, cand_rid, &s_misc[0]);
        if (c >= kk && c <= BT_CAND) {
            cand = true;
            src_n = c;
            const int lz = __clzll(static_cast<long long>(t));
            L = lz < kb ? lz : kb;
        }
    }
    // Block-local radix refine of the (rank word, row-id) prefix.
    uint64_t p0 = 0, p1 = 0, krem = kk, bcnt = src_n;
    const unsigned lane = threadIdx.x & 31u;
    while (bcnt > BT_SMALL && L < TB && krem < bcnt) {
        const int d = min(digit, TB - L);
        for (int b = threadIdx.x; b < BT_BINS; b += BT_TPB) hist[b] = 0;
        __syncthreads();
        for (uint64_t wb = threadIdx.x & ~31u; wb < src_n; wb += BT_TPB) {
            const uint64_t i = wb + lane;
            unsigned dig = 0xFFFFFFFFu;
            if (i < src_n) {
                uint64_t r;
                uint32_t rid;
                src_get(it, cand, cand_r, cand_rid, i, r, rid);
                uint64_t w0, w1;
                comp_words(r, rid, kb, w0, w1);
                if (prefix_cmp(w0, w1, p0, p1, L) == 0) dig = comp_digit(w0, w1, L, d);
            }
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
            if (dig != 0xFFFFFFFFu && lane == static_cast<unsigned>(__ffs(peers) - 1))
                atomicAdd(&hist[dig], static_cast<unsigned>(__popc(peers)));
        }
        __syncthreads();
        const Pick pk = pick_bucket<BT_TPB>(hist, krem, sc);
        krem -= pk.below;
        bcnt = pk.in_b;
        prefix_set(p0, p1, L, d, pk.b);
        L += d;
    }
    // Split: below-prefix entries to sr[0, nb), prefix-equal ones to
    // sr[BT_SMALL, ...) (or straight after the below ones when all of them,
    // or any krem identical ones, are taken).
    const bool take_all = (krem == bcnt) || (L >= TB);
    const uint64_t nb = kk - krem;
    unsigned* s_below = &s_misc[1];
    unsigned* s_eq = &s_misc[2];
    if (threadIdx.x == 0) {
        *s_below = 0;
        *s_eq = 0;
    }
    __syncthreads();
    for (uint64_t wb = threadIdx.x & ~31u; wb < src_n; wb += BT_TPB) {
        const uint64_t i = wb + lane;
        int c = 1;
        uint64_t r = 0;
        uint32_t rid = 0;
        if (i < src_n) {
            src_get(it, cand, cand_r, cand_rid, i, r, rid);
            uint64_t w0, w1;
            comp_words(r, rid, kb, w0, w1);
            c = prefix_cmp(w0, w1, p0, p1, L);
        }
        if (c < 0) {
            const unsigned pos = atomicAdd(s_below, 1u);
            sr[pos] = r;
            srid[pos] = rid;
        } else if (c == 0) {
            const unsigned pos = atomicAdd(s_eq, 1u);
            if (take_all) {
                if (pos < krem) {
                    sr[nb + pos] = r;
                    srid[nb + pos] = rid;
                }
            } else if (pos < BT_SMALL) {
                sr[BT_SMALL + pos] = r;
                srid[BT_SMALL + pos] = rid;
            }
        }
    }
    __syncthreads();
    // Finish: sort the selected entries and write them out.
    if (take_all) {
        block_sort<BT_TPB>(sr, srid, static_cast<int>(kk));
        for (uint64_t i = threadIdx.x; i < kk; i += BT_TPB) put_result(it, i, sr[i], srid[i]);
    } else {
        block_sort<BT_TPB>(sr + BT_SMALL, srid + BT_SMALL, static_cast<int>(bcnt));
        block_sort<BT_TPB>(sr, srid, static_cast<int>(nb));
        for (uint64_t i = threadIdx.x; i < nb; i += BT_TPB) put_result(it, i, sr[i], srid[i]);
        for (uint64_t i = threadIdx.x; i < krem; i += BT_TPB) put_result(it, nb + i, sr[BT_SMALL + i], srid[BT_SMALL + i]);
    }
    if (threadIdx.x == 0) *it.count = kk;
}

// Device-side check of a work descriptor; OLAP_OK when it can run.
__device__ int item_check(const Item& it) {
    if (it.op != OLAP_OP_TOPK && it.op != OLAP_OP_PROBE) return OLAP_E_DEVICE;
    if (!it.count) return OLAP_E_DEVICE;
    if (it.n && !it.keys) return OLAP_E_DEVICE;
    if (it.n >= (1ull << 32)) return OLAP_E_DEVICE;
    if (it.op == OLAP_OP_TOPK) {
        if (it.k > BT_SMALL) return OLAP_E_DEVICE;
        if (it.k && it.n && (!it.out_keys || !it.out_rowids)) return OLAP_E_DEVICE;
        if (it.kind < OLAP_KEY_I64 || it.kind > OLAP_KEY_U32 || it.w4 != (key_bytes(it.kind) == 4))
            return OLAP_E_DEVICE;
        if (reinterpret_cast<uintptr_t>(it.keys) % (it.w4 ? 4 : 8)) return OLAP_E_DEVICE;
    } else {
        if (!it.table || ((it.mask + 1) & it.mask)) return OLAP_E_DEVICE;
        if (it.cap && !it.out_pairs) return OLAP_E_DEVICE;
        if (it.n_side && !it.side) return OLAP_E_DEVICE;
    }
    return OLAP_OK;
}

// Persistent Top-K executor: each CTA takes the next Top-K item off the queue.
__global__ void __launch_bounds__(BT_TPB, 2) batch_topk_kernel(const Item* items, uint64_t n_items,
                                                               unsigned long long* next, uint64_t* cand_r_all,
                                                               uint32_t* cand_rid_all, int* errors, int digit) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long sc[24];
    __shared__ unsigned s_misc[4];
    __shared__ unsigned long long s_item;
    __shared__ Item s_it;
    uint64_t* cand_r = cand_r_all + static_cast<uint64_t>(blockIdx.x) * BT_CAND;
    uint32_t* cand_rid = cand_rid_all + static_cast<uint64_t>(blockIdx.x) * BT_CAND;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(next, 1ull);
        __syncthreads();
        const uint64_t idx = s_item;
        if (idx >= n_items) break;
        if (threadIdx.x < sizeof(Item) / 8)
            reinterpret_cast<uint64_t*>(&s_it)[threadIdx.x] = reinterpret_cast<const uint64_t*>(items + idx)[threadIdx.x];
        __syncthreads();
        const Item& it = s_it;
        const int st = it.op == OLAP_OP_TOPK ? item_check(it) : static_cast<int>(OLAP_E_DEVICE);
        if (st == OLAP_OK) cta_topk(it, smem, cand_r, cand_rid, sc, s_misc, digit);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (it.status) *it.status = st;
            if (st != OLAP_OK) atomicAdd(errors, 1);
        }
        __syncthreads();
    }
}

// Before the probe queue starts: check each probe item, zero its pair count
// and record its status (one thread per item).
__global__ void batch_probe_reset_kernel(const Item* items, uint64_t n_items, int* errors) {
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    const Item& it = items[i];
    const int st = it.op == OLAP_OP_PROBE ? item_check(it) : static_cast<int>(OLAP_E_DEVICE);
    if (st == OLAP_OK) *it.count = 0;
    if (it.status) *it.status = st;
    if (st != OLAP_OK) atomicAdd(errors, 1);
}

// Persistent probe executor: each CTA takes the next chunk off the queue and
// splits its rows over its warps; chunks of items that failed the check are
// skipped.
__global__ void __launch_bounds__(JP_TPB, 3) batch_probe_kernel(const Item* items, const ProbeChunk* chunks,
                                                                uint64_t n_chunks, unsigned long long* next) {
    extern __shared__ __align__(16) uint2 stage[];
    __shared__ unsigned long long s_item;
    __shared__ ProbeChunk s_ch;
    __shared__ int s_ok;
    __shared__ ProbeArgs s_args;       // kept in shared memory, read as needed
    __shared__ unsigned long long s_next;   // the chunk's row queue, shared by the CTA's warps
    uint32_t cur = 0xFFFFFFFFu;        // item whose arguments s_args holds
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(next, 1ull);
        __syncthreads();
        const uint64_t idx = s_item;
        if (idx >= n_chunks) break;
        if (threadIdx.x == 0) {
            s_ch = chunks[idx];
            if (s_ch.item != cur) {
                const Item& it = items[s_ch.item];
                s_ok = it.op == OLAP_OP_PROBE && item_check(it) == OLAP_OK;
                s_args.keys = static_cast<const int64_t*>(it.keys);
                s_args.rowids = it.rowids;
                s_args.n = it.n;
                s_args.slots = reinterpret_cast<const ulonglong2*>(it.table);
                s_args.mask = it.mask;
                s_args.side = it.side;
                s_args.n_side = it.n_side;
                s_args.out = it.out_pairs;
                s_args.cap = it.cap;
                s_args.count = it.count;
            }
            s_next = static_cast<uint64_t>(s_ch.chunk) * BP_CHUNK;
        }
        __syncthreads();
        cur = s_ch.item;
        if (s_ok) {
            // the chunk's rows go to the CTA's warps through a row queue in
            // shared memory (the probe loop of the join kernel)
            RowQueue q;
            q.counter = &s_next;
            q.n = min(s_args.n, static_cast<uint64_t>(s_ch.chunk) * BP_CHUNK + BP_CHUNK);
            probe_queue<true, JP_S>(s_args, q, stage + (threadIdx.x >> 5) * JP_WCAP);
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace olap

using namespace olap;

struct olap_batch {
    olap_ctx* ctx = nullptr;
    std::vector<olap_batch_item> items;   // caller's order (per-query baseline)
    Item* d_items = nullptr;              // Top-K items then probe items, each largest first
    uint64_t n_topk = 0, n_probe = 0;
    ProbeChunk* d_chunks = nullptr;       // probe work units, largest items first
    uint64_t n_chunks = 0;
    unsigned long long* d_next = nullptr; // [0] Top-K queue head, [8] probe queue head
    int* d_errors = nullptr;
    uint64_t* cand_r = nullptr;
    uint32_t* cand_rid = nullptr;
    // Split Top-K items: the merge items (run after the first Top-K launch)
    // and the parts' results (rank words, row-ids, counts).
    Item* d_merge = nullptr;
    uint64_t n_merge = 0;
    void* part_buf = nullptr;
    int grid_topk = 0, grid_probe = 0;
    // Overlap: the probe branch runs on a second stream forked from the
    // launch stream inside the graph (the two kernels are independent).
    bool overlap = false;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int digit = 12;                       // radix digit width of the per-CTA Top-K
    int graph_kernels = 0;                // kernels in the captured graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

olap_status enqueue_batch(olap_batch* b, cudaStream_t s) {
    // queue heads and the error count live in one 256-byte block
    cudaError_t e = cudaMemsetAsync(b->d_next, 0, 256, s);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "batch reset");
    cudaStream_t ps = s;                      // stream of the probe branch
    if (b->overlap) {
        if ((e = cudaEventRecord(b->ev_fork, s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(b->side, b->ev_fork, 0)) != cudaSuccess)
            return cuda_fail(b->ctx, e, "batch fork");
        ps = b->side;
    }
    b->graph_kernels = 0;
    if (b->n_probe) {
        const Item* probe_items = b->d_items + b->n_topk;
        batch_probe_reset_kernel<<<static_cast<unsigned>((b->n_probe + 255) / 256), 256, 0, ps>>>(
            probe_items, b->n_probe, b->d_errors);
        ++b->graph_kernels;
        if (b->n_chunks) {
            batch_probe_kernel<<<b->grid_probe, JP_TPB, JP_SMEM, ps>>>(probe_items, b->d_chunks, b->n_chunks,
                                                                       b->d_next + 1);
            ++b->graph_kernels;
        }
    }
    if (b->n_topk) {
        batch_topk_kernel<<<b->grid_topk, BT_TPB, BT_SMEM, s>>>(b->d_items, b->n_topk, b->d_next, b->cand_r,
                                                                b->cand_rid, b->d_errors, b->digit);
        ++b->graph_kernels;
    }
    if (b->n_merge) {          // after every part: the merges of split items
        const unsigned mg = static_cast<unsigned>(std::min<uint64_t>(b->n_merge, b->grid_topk));
        batch_topk_kernel<<<mg, BT_TPB, BT_SMEM, s>>>(b->d_merge, b->n_merge, b->d_next + 2, b->cand_r,
                                                      b->cand_rid, b->d_errors, b->digit);
        ++b->graph_kernels;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(b->ctx, e, "batch launch");
    if (b->overlap &&
        ((e = cudaEventRecord(b->ev_join, b->side)) != cudaSuccess || (e = cudaStreamWaitEvent(s, b->ev_join, 0)) !=
                                                                         cudaSuccess))
        return cuda_fail(b->ctx, e, "batch join");
    return OLAP_OK;
}

void batch_release(olap_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_merge) cudaFree(b->d_merge);
    if (b->part_buf) cudaFree(b->part_buf);
    if (b->d_chunks) cudaFree(b->d_chunks);
    if (b->d_next) cudaFree(b->d_next);
    if (b->cand_r) cudaFree(b->cand_r);
    if (b->cand_rid) cudaFree(b->cand_rid);
    delete b;
}

}  // namespace

extern "C" {

olap_status olap_batch_create(olap_ctx* ctx, const olap_batch_item* items, uint64_t n_items, olap_batch** out) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!out || (n_items && !items)) return fail(ctx, OLAP_E_INVALID, "NULL argument");
    *out = nullptr;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");
    std::vector<Item> dev(n_items);
    std::vector<double> cost(n_items);
    for (uint64_t i = 0; i < n_items; ++i) {
        const olap_batch_item& x = items[i];
        Item& d = dev[i];
        std::memset(&d, 0, sizeof(d));
        d.op = x.op;
        d.keys = x.keys;
        d.rowids = x.rowids;
        d.n = x.n;
        d.count = reinterpret_cast<unsigned long long*>(x.count);
        d.status = x.status;
        if (x.op == OLAP_OP_TOPK) {
            if (x.key_type < OLAP_KEY_I64 || x.key_type > OLAP_KEY_U32)
                return fail(ctx, OLAP_E_INVALID, "batch item: bad key type");
            if (x.k > BT_SMALL) return fail(ctx, OLAP_E_INVALID, "batch item: Top-K k above 4096 (use olap_topk)");
            d.kind = x.key_type;
            d.w4 = key_bytes(x.key_type) == 4;
            d.desc = x.order == OLAP_DESC;
            d.k = x.k;
            d.out_keys = x.out_keys;
            d.out_rowids = x.out_rowids;
            cost[i] = static_cast<double>(x.n) * (d.w4 ? 4.0 : 8.0);
        } else if (x.op == OLAP_OP_PROBE) {
            if (!x.table || !x.table->slots) return fail(ctx, OLAP_E_INVALID, "batch item: NULL join table");
            if (x.table->device != ctx->device) return fail(ctx, OLAP_E_INVALID, "batch item: table on another device");
            d.table = reinterpret_cast<const uint64_t*>(x.table->slots);
            d.mask = x.table->n_buckets - 1;
            d.side = x.table->side;
            d.n_side = x.table->n_side;
            d.out_pairs = reinterpret_cast<uint2*>(x.out_pairs);
            d.cap = x.capacity;
            cost[i] = static_cast<double>(x.n) * 48.0;
        } else {
            return fail(ctx, OLAP_E_INVALID, "batch item: bad op");
        }
        if (!x.count) return fail(ctx, OLAP_E_INVALID, "batch item: NULL count");
        if (x.n >= (1ull << 32)) return fail(ctx, OLAP_E_INVALID, "batch item: n must be below 2^32");
    }
    // Top-K items first, then probe items; each group largest first, so the
    // long items start early and short ones fill in.
    std::vector<uint64_t> order(n_items);
    std::iota(order.begin(), order.end(), 0ull);
    std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) {
        if (dev[a].op != dev[b].op) return dev[a].op == OLAP_OP_TOPK;
        return cost[a] > cost[b];
    });
    // A Top-K item larger than one CTA's share of the batch's Top-K bytes
    // would keep its CTA busy after the others run dry (the items are
    // scheduled largest first, so smaller ones balance the rest).  Such an
    // item is split into parts of about that share (at least BT_PART rows):
    // each part selects its own Top-K (rank words and row-ids into part_buf)
    // and a merge item selects the item's Top-K from the parts' results in a
    // second launch.  Measured on the 4096-query batch, where no item exceeds
    // the share, splitting every item above 2^19 keys was slower (8.0 against
    // 6.3 ms): the parts' fixed costs outweigh a tail that is not there.
    const int topk_ctas_hint = ctx->sm_count * 2;
    double topk_bytes = 0.0;
    for (uint64_t i = 0; i < n_items; ++i)
        if (dev[i].op == OLAP_OP_TOPK) topk_bytes += static_cast<double>(dev[i].n) * (dev[i].w4 ? 4.0 : 8.0);
    const double share = topk_bytes / std::max(1, topk_ctas_hint);
    struct Split {
        uint64_t item, parts, len;
    };
    std::vector<Split> splits;
    uint64_t part_entries = 0;
    for (uint64_t i = 0; i < n_items; ++i) {
        const Item& d = dev[i];
        const size_t w = d.w4 ? 4 : 8;
        if (d.op != OLAP_OP_TOPK || d.n < BT_SPLIT_N || d.k == 0 || reinterpret_cast<uintptr_t>(d.keys) % w ||
            static_cast<double>(d.n) * w <= share)
            continue;
        const uint64_t part = std::max<uint64_t>(BT_PART, static_cast<uint64_t>(share / w));
        const uint64_t parts = (d.n + part - 1) / part;
        if (parts < 2) continue;
        splits.push_back({i, parts, (d.n + parts - 1) / parts});
        part_entries += parts * d.k;
    }
    std::vector<Item> topk_units, merges;
    void* part_buf = nullptr;
    if (!splits.empty()) {
        // [rank words | row-ids | counts], each 256-byte aligned
        const size_t rb = (part_entries * 8 + 255) & ~static_cast<size_t>(255);
        const size_t ib = (part_entries * 4 + 255) & ~static_cast<size_t>(255);
        e = cudaMalloc(&part_buf, rb + ib + splits.size() * 8);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(ctx, e, "batch part results");
        }
        unsigned char* pb = static_cast<unsigned char*>(part_buf);
        uint64_t* ranks = reinterpret_cast<uint64_t*>(pb);
        uint32_t* rids = reinterpret_cast<uint32_t*>(pb + rb);
        unsigned long long* counts = reinterpret_cast<unsigned long long*>(pb + rb + ib);
        uint64_t at = 0, nc = 0;
        for (const Split& sp : splits) {
            Item& orig = dev[sp.item];
            const size_t w = orig.w4 ? 4 : 8;
            for (uint64_t p = 0; p < sp.parts; ++p) {
                Item part = orig;
                const uint64_t off = p * sp.len;
                part.keys = static_cast<const unsigned char*>(orig.keys) + off * w;
                part.rowids = orig.rowids ? orig.rowids + off : nullptr;
                part.rowid_base = orig.rowids ? 0 : off;
                part.n = std::min(sp.len, orig.n - off);
                part.out_mode = ITEM_OUT_RANKS;
                part.out_keys = ranks + at + p * orig.k;
                part.out_rowids = rids + at + p * orig.k;
                part.count = counts + nc;                    // parts share one scratch count word per item
                part.status = nullptr;
                topk_units.push_back(part);
            }
            Item m = orig;
            m.kind = OLAP_KEY_U64;
            m.w4 = 0;
            m.desc = 0;
            m.keys = ranks + at;
            m.rowids = rids + at;
            m.rowid_base = 0;
            m.n = sp.parts * orig.k;
            m.out_mode = ITEM_OUT_MERGE;
            m.out_kind = orig.kind;
            m.out_desc = orig.desc;
            merges.push_back(m);
            at += sp.parts * orig.k;
            nc += 1;
            orig.op = -1;                                    // replaced by its parts and merge
        }
    }
    std::vector<Item> sorted;
    sorted.reserve(n_items + topk_units.size());
    for (uint64_t i = 0; i < n_items; ++i)
        if (dev[order[i]].op == OLAP_OP_TOPK) topk_units.push_back(dev[order[i]]);
    std::stable_sort(topk_units.begin(), topk_units.end(),
                     [](const Item& a, const Item& b) { return a.n * (a.w4 ? 4 : 8) > b.n * (b.w4 ? 4 : 8); });
    const uint64_t n_topk = topk_units.size();
    sorted = topk_units;
    for (uint64_t i = 0; i < n_items; ++i)
        if (dev[order[i]].op == OLAP_OP_PROBE) sorted.push_back(dev[order[i]]);
    const uint64_t n_units = sorted.size();

    // Probe work units: each item cut into chunks of BP_CHUNK rows, in the
    // items' (largest first) order.
    std::vector<ProbeChunk> chunks;
    for (uint64_t i = n_topk; i < n_units; ++i) {
        const uint64_t nch = (sorted[i].n + BP_CHUNK - 1) / BP_CHUNK;
        for (uint64_t c = 0; c < nch; ++c)
            chunks.push_back({static_cast<uint32_t>(i - n_topk), static_cast<uint32_t>(c)});
    }

    olap_batch* b = new olap_batch();
    b->ctx = ctx;
    b->digit = ctx->opts.topk_digit_bits ? ctx->opts.topk_digit_bits : 12;
    b->n_chunks = chunks.size();
    b->items.assign(items, items + n_items);
    b->n_topk = n_topk;
    b->n_probe = n_units - n_topk;
    b->part_buf = part_buf;
    b->n_merge = merges.size();
    int per_t = 0, per_p = 0;
    if ((e = cudaFuncSetAttribute(batch_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(batch_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, JP_SMEM)) !=
            cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_t, batch_topk_kernel, BT_TPB, BT_SMEM)) !=
            cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_p, batch_probe_kernel, JP_TPB, JP_SMEM)) !=
            cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        return cuda_fail(ctx, e, "batch kernel set-up");
    }
    const int topk_per_sm = ctx->opts.batch_topk_ctas_per_sm > 0 ? ctx->opts.batch_topk_ctas_per_sm : 2;
    b->grid_topk = ctx->sm_count * std::max(1, std::min(per_t, topk_per_sm));
    b->overlap = ctx->opts.batch_overlap == 1 && n_topk > 0 && n_units > n_topk;
    if (b->overlap &&
        ((e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess ||
         (e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
         (e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming)) != cudaSuccess)) {
        cudaGetLastError();
        batch_release(b);
        return cuda_fail(ctx, e, "batch streams");
    }
    b->grid_probe = ctx->sm_count * std::max(1, per_p);
    if ((e = cudaMalloc(&b->d_items, std::max<uint64_t>(1, n_units) * sizeof(Item))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_merge, std::max<size_t>(1, merges.size()) * sizeof(Item))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_chunks, std::max<size_t>(1, chunks.size()) * sizeof(ProbeChunk))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&b->d_next), 256)) != cudaSuccess ||
        (e = cudaMalloc(&b->cand_r, static_cast<size_t>(b->grid_topk) * BT_CAND * 8)) != cudaSuccess ||
        (e = cudaMalloc(&b->cand_rid, static_cast<size_t>(b->grid_topk) * BT_CAND * 4)) != cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        return cuda_fail(ctx, e, "batch allocation");
    }
    b->d_errors = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(b->d_next) + 64);

    if ((n_units && (e = cudaMemcpy(b->d_items, sorted.data(), n_units * sizeof(Item), cudaMemcpyHostToDevice)) !=
                        cudaSuccess) ||
        (!merges.empty() && (e = cudaMemcpy(b->d_merge, merges.data(), merges.size() * sizeof(Item),
                                            cudaMemcpyHostToDevice)) != cudaSuccess)) {
        batch_release(b);
        return cuda_fail(ctx, e, "batch descriptor upload");
    }
    if (!chunks.empty() && (e = cudaMemcpy(b->d_chunks, chunks.data(), chunks.size() * sizeof(ProbeChunk),
                                           cudaMemcpyHostToDevice)) != cudaSuccess) {
        batch_release(b);
        return cuda_fail(ctx, e, "batch chunk upload");
    }
    // Capture the reset and the persistent launch in a CUDA graph.
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_release(b);
        return cuda_fail(ctx, e, "capture stream");
    }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    olap_status st = e == cudaSuccess ? enqueue_batch(b, cap) : cuda_fail(ctx, e, "begin capture");
    cudaError_t e2 = cudaStreamEndCapture(cap, &b->graph);
    cudaStreamDestroy(cap);
    if (st != OLAP_OK || e2 != cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        return st != OLAP_OK ? st : cuda_fail(ctx, e2, "end capture");
    }
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
        cudaGetLastError();
        batch_release(b);
        return cuda_fail(ctx, e, "graph instantiate");
    }
    *out = b;
    return OLAP_OK;
}

olap_status olap_batch_run(olap_batch* b, void* stream) {
    if (!b) return OLAP_E_INVALID;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->ctx->stream;
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "batch graph launch");
    b->ctx->launches += static_cast<uint64_t>(b->graph_kernels);
    return OLAP_OK;
}

olap_status olap_batch_run_per_query(olap_batch* b, void* stream) {
    if (!b) return OLAP_E_INVALID;
    olap_ctx* ctx = b->ctx;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    for (const olap_batch_item& x : b->items) {
        olap_status st;
        if (x.op == OLAP_OP_TOPK) {
            st = olap_topk_async(ctx, x.keys, static_cast<olap_key_type>(x.key_type), x.rowids, x.n, x.k,
                                 static_cast<olap_order>(x.order), x.out_keys, x.out_rowids, x.status, s);
        } else {
            st = olap_join_probe_async(ctx, x.table, static_cast<const int64_t*>(x.keys), x.rowids, x.n,
                                       x.out_pairs, x.capacity, x.count, s);
        }
        if (st != OLAP_OK) return st;
    }
    return OLAP_OK;
}

olap_status olap_batch_errors(olap_batch* b, int* errors) {
    if (!b || !errors) return OLAP_E_INVALID;
    cudaError_t e = cudaStreamSynchronize(b->ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(errors, b->d_errors, sizeof(int), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? OLAP_OK : cuda_fail(b->ctx, e, "batch errors read-back");
}

void olap_batch_free(olap_batch* b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    batch_release(b);
}

}  // extern "C"
