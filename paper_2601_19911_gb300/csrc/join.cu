// Key-based hash join over key-only columns (Sec. III-B: "parallel probing
// using a key-only hash table"; pointers returned for late materialization,
// Sec. II-C).
//
// Table: open addressing, 16-byte slots {int64 key, row-id}, two slots per
// 32-byte bucket (one DRAM sector), linear probing over buckets.  A key goes
// to the first free slot at or after its home bucket, slot 0 before slot 1,
// so a bucket with a free slot ends every chain.  The empty marker is the key
// with all bits set; build rows carrying that key value live in a side list.
// Hash: the 64-bit finalizer of MurmurHash3 (fmix64, A. Appleby).
//
// Build: one CAS pass, then a pass that records in every occupied slot how
// many further copies of its key follow it along the chain, so a probe can
// stop at a key's last copy instead of walking on to the chain's end.
//
// Probe: every warp takes chunks of consecutive rows from a global counter
// and hands them to its lanes in order (the loads of keys and row-ids
// coalesce; no lane waits at a partition or range boundary).  Each lane runs
// two independent probe streams and walks their chains one bucket per step; a
// stream whose chain ends starts its next row at once (its key is already
// loaded), so lanes do not wait for the longest chain of the warp.  Matches
// are staged per warp in shared memory and appended to the output with one
// atomic on the global count per flush.
//
// Partitioned probe (table much larger than L2, many probe rows): a table
// larger than L2 turns every probe into a random DRAM sector read, and those
// run at a small fraction of the streaming rate.  Instead the probe rows are
// first radix-partitioned by the top bits of their home bucket into P
// partitions (a counting pass and a scatter pass, both streaming, with the
// same CTA-to-tile assignment so every CTA's output ranges come from the
// count matrix without global atomics).  The probe then takes the reordered
// rows chunk by chunk in partition order, so the whole grid works on one
// 1/P slice of the table at a time, sized to stay resident in L2: the table
// is read from DRAM about once.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>

#include "block.cuh"
#include "ctx.h"
#include "join_dev.cuh"

namespace olap {

namespace {

__global__ void __launch_bounds__(JB_TPB) join_build_kernel(const int64_t* keys, const uint32_t* rowids,
                                                            uint64_t n, ulonglong2* slots, uint64_t mask,
                                                            JoinCtl* ctl) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * JB_TPB;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * JB_TPB + threadIdx.x; i < n; i += stride) {
        const uint64_t key = static_cast<uint64_t>(keys[i]);
        if (key == JN_EMPTY) {
            atomicAdd(&ctl->side_count, 1ull);
            continue;
        }
        const uint32_t rid = rowids ? rowids[i] : static_cast<uint32_t>(i);
        uint64_t b = fmix64(key) & mask;
        bool done = false;
        for (uint64_t step = 0; step <= mask && !done; ++step) {
            for (int s = 0; s < 2 && !done; ++s) {
                unsigned long long* kp = reinterpret_cast<unsigned long long*>(&slots[b * 2 + s].x);
                if (*reinterpret_cast<volatile unsigned long long*>(kp) != JN_EMPTY) continue;
                if (atomicCAS(kp, JN_EMPTY, static_cast<unsigned long long>(key)) == JN_EMPTY) {
                    slots[b * 2 + s].y = rid;
                    done = true;
                }
            }
            b = (b + 1) & mask;
        }
        if (!done) atomicCAS(&ctl->err, 0, static_cast<int>(OLAP_E_DEVICE));
    }
}

// After the build: every occupied slot records, in the high half of its
// row-id word, how many further copies of its key follow it along the chain
// (up to the first bucket with a free slot, where every chain through it
// ends).  Copies of a key all sit between its home bucket and that end, in
// the order a probe walks them, so a probe that meets a copy with no further
// copies has seen them all and stops there instead of walking to the chain's
// end: for a unique build a hit stops at its key.
__global__ void __launch_bounds__(JB_TPB) join_chain_kernel(ulonglong2* slots, uint64_t mask) {
    const uint64_t n_slots = (mask + 1) * 2;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * JB_TPB;
    for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * JB_TPB + threadIdx.x; j < n_slots; j += stride) {
        const uint64_t key = slots[j].x;
        if (key == JN_EMPTY) continue;
        uint64_t b = j >> 1;
        uint32_t further = 0;
        uint64_t k1 = slots[b * 2 + 1].x;
        if ((j & 1) == 0 && k1 == key) ++further;
        for (uint64_t step = 0; k1 != JN_EMPTY && step < mask; ++step) {   // bucket b full: the chain goes on
            b = (b + 1) & mask;
            const uint64_t k0 = slots[b * 2].x;
            k1 = slots[b * 2 + 1].x;
            further += (k0 == key) + (k1 == key);
        }
        slots[j].y = (slots[j].y & 0xFFFFFFFFull) | (static_cast<uint64_t>(further) << 32);
    }
}

__global__ void __launch_bounds__(JB_TPB) join_side_kernel(const int64_t* keys, const uint32_t* rowids,
                                                           uint64_t n, uint32_t* side, JoinCtl* ctl) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * JB_TPB;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * JB_TPB + threadIdx.x; i < n; i += stride) {
        if (static_cast<uint64_t>(keys[i]) == JN_EMPTY) {
            const unsigned long long pos = atomicAdd(&ctl->side_fill, 1ull);
            side[pos] = rowids ? rowids[i] : static_cast<uint32_t>(i);
        }
    }
}

// The probe: rows [0, a.n) handed out in chunks by a row queue (see
// probe_queue).  Used on the input (direct probe) and on the rows reordered
// by partition (pass 3 of the partitioned probe): there the chunks come out in
// partition order, so the warps of the whole grid work on one partition's
// table slice at a time and that slice stays in L2.
// `args` holds the rows as launched (the probe's input, or its partitioned
// rows).  The device-side plan (ctl, when non-NULL) may change that: with the
// Bloom pre-probe active the row count is the number of rows it kept, and
// with `redirect` the rows are read from where the plan says (the kept rows,
// or the input when the partition passes were skipped), through L1 when the
// plan says so.
template <bool L2_ONLY>
__global__ void __launch_bounds__(JP_TPB, 4) join_probe_kernel(ProbeArgs args, unsigned long long* next_row,
                                                               const ProbeCtl* ctl) {
    extern __shared__ __align__(16) uint2 stage[];
    const unsigned warp = threadIdx.x >> 5;
    ProbeArgs a = args;
    bool l1 = !L2_ONLY;
    if (ctl) {
        if (ctl->active) a.n = ctl->count;
        if (ctl->redirect) {
            a.keys = ctl->keys;
            a.rowids = ctl->rowids;
        }
        l1 = l1 || ctl->l1;
    }
    RowQueue q;
    q.counter = next_row;
    q.n = a.n;
    if (l1)
        probe_queue<false, JP_S>(a, q, stage + warp * JP_WCAP);
    else
        probe_queue<true, JP_S>(a, q, stage + warp * JP_WCAP);
}

// ---- Bloom pre-probe ------------------------------------------------------

// Every build key sets its eight bits in its block (the empty-marker key,
// kept in the side list, is not entered: the pre-probe keeps such probe rows
// whatever the filter says).
__global__ void __launch_bounds__(JB_TPB) join_bloom_kernel(const int64_t* keys, uint64_t n, uint32_t* bloom,
                                                            uint64_t bmask) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * JB_TPB;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * JB_TPB + threadIdx.x; i < n; i += stride) {
        const uint64_t key = static_cast<uint64_t>(keys[i]);
        if (key == JN_EMPTY) continue;
        uint32_t* blk = bloom + bloom_block(key, bmask) * BLOOM_WORDS;
        const uint64_t g = fmix64(~key);
#pragma unroll
        for (int w = 0; w < BLOOM_WORDS; ++w) atomicOr(blk + w, bloom_bit(g, w));
    }
}

constexpr int PF_TPB = 256;
constexpr int PF_SAMPLE = 4096;                // probe keys tested to decide
constexpr uint64_t PF_MIN_N = 1ull << 20;      // smaller probes skip the pre-probe (automatic mode)
constexpr int PF_PER = 4;                      // keys per lane per step
constexpr unsigned PF_WCAP = 256;              // rows staged per warp

constexpr int PLAN_SLOTS = 2 * PF_SAMPLE;      // fingerprint set of the sample (32 KB)
constexpr int PLAN_CTAS = PF_SAMPLE / PF_TPB;  // one sampled key per thread

// The plan kernel's inputs, and its state in the context's device area.
struct PlanArgs {
    const int64_t* keys;
    const uint32_t* rowids;
    uint64_t n;
    const uint32_t* bloom;                     // NULL: no pre-probe stage
    uint64_t bmask;
    int pf_mode;                               // 1 automatic, 2 forced (with a filter)
    int skew_check;
    int partitioned;
    int skew_l1;
    const int64_t* pf_keys;
    const uint32_t* pf_rowids;
    uint32_t* sample;                          // PF_SAMPLE packed entries
    unsigned* counters;                        // [0] kept keys, [1] CTAs done; zero between calls
    ProbeCtl* ctl;
};

// The probe's plan, decided on the device from a stratified sample of
// PF_SAMPLE probe keys (n >= PF_SAMPLE; fewer rows are each taken once or
// more).  PLAN_CTAS CTAs load the sample, one key per thread (from one SM,
// 4096 scattered loads wait on each other's latency: 38 us), test it
// against the Bloom filter and store one packed word per key: a 30-bit
// fingerprint of the key, bit 1 = kept by the filter, bit 0 = 1.  The last
// CTA to finish decides.  With a Bloom filter (pf_mode 1 = automatic,
// 2 = forced) the pre-probe runs when at most 60 % of the sample may be in
// the table, or always when forced.  With `skew_check` the probe skips its
// partition passes when the rows it will probe repeat: at least a fifth of
// the sampled keys that reach the probe (those the filter keeps, when it
// runs) equal an earlier sampled key.  Such a stream sends most probes to a
// few hot buckets, which stay in cache, while the partition passes would
// cost two more passes over the rows.  Repeats are found in a shared-memory
// fingerprint set; a fingerprint collision counts as a repeat (about 2^-7
// of one per sample).  The last CTA zeroes the kept-row count and tells the
// probe kernel where its rows are: the partitioned rows (`partitioned` and
// not direct, as launched), else the kept rows (pf_keys, pf_rowids) when the
// pre-probe runs, else the input; a direct probe reads buckets through L1
// when `skew_l1`.  It also clears the counters for the next call.
__global__ void __launch_bounds__(PF_TPB) join_probe_plan_kernel(PlanArgs a) {
    __shared__ uint32_t fset[PLAN_SLOTS];
    __shared__ unsigned kept_cta, dup_all, dup_kept;
    __shared__ bool last;
    if (threadIdx.x == 0) kept_cta = 0;
    __syncthreads();
    {
        const uint64_t j = static_cast<uint64_t>(blockIdx.x) * PF_TPB + threadIdx.x;     // < PF_SAMPLE
        const uint64_t key = static_cast<uint64_t>(a.keys[(j * a.n) / PF_SAMPLE]);
        const bool kept = a.bloom ? (key == JN_EMPTY || bloom_maybe(a.bloom, a.bmask, key)) : true;
        const uint32_t fp = static_cast<uint32_t>(fmix64(key) >> 32) & ~3u;
        a.sample[j] = fp | (kept ? 2u : 0u) | 1u;
        if (kept) atomicAdd(&kept_cta, 1u);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&a.counters[0], kept_cta);
        last = atomicAdd(&a.counters[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = threadIdx.x; j < PLAN_SLOTS; j += PF_TPB) fset[j] = 0u;
    if (threadIdx.x == 0) dup_all = dup_kept = 0;
    __syncthreads();
    unsigned m_dup = 0, m_dup_kept = 0;
    if (a.skew_check) {
        for (int j = threadIdx.x; j < PF_SAMPLE; j += PF_TPB) {
            const uint32_t w = __ldcg(a.sample + j);
            const uint32_t fp = w & ~2u;                 // the fingerprint, with the set's non-zero bit
            uint32_t slot = (fp >> 2) & (PLAN_SLOTS - 1);
            bool dup = false;
            for (int tries = 0; tries < PLAN_SLOTS; ++tries) {
                const uint32_t prev = atomicCAS(&fset[slot], 0u, fp);
                if (prev == 0u) break;
                if (prev == fp) {
                    dup = true;
                    break;
                }
                slot = (slot + 1) & (PLAN_SLOTS - 1);
            }
            m_dup += dup ? 1u : 0u;
            m_dup_kept += (dup && (w & 2u)) ? 1u : 0u;
        }
    }
    atomicAdd(&dup_all, m_dup);
    atomicAdd(&dup_kept, m_dup_kept);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned passes = atomicAdd(&a.counters[0], 0u);
        const bool active = a.bloom && (a.pf_mode == 2 || passes * 10u <= static_cast<unsigned>(PF_SAMPLE) * 6u);
        const unsigned reach = active ? passes : static_cast<unsigned>(PF_SAMPLE);
        const unsigned rep = active ? dup_kept : dup_all;
        const bool direct = a.skew_check && reach >= 64u && rep * 5u >= reach;
        ProbeCtl* ctl = a.ctl;
        ctl->active = active ? 1 : 0;
        ctl->direct = direct ? 1 : 0;
        ctl->count = 0;
        ctl->redirect = (!a.partitioned || direct) ? 1 : 0;
        ctl->keys = active ? a.pf_keys : a.keys;
        ctl->rowids = active ? a.pf_rowids : a.rowids;
        ctl->l1 = (direct && a.skew_l1) ? 1 : 0;
        a.counters[0] = 0;
        a.counters[1] = 0;
    }
}

// The pre-probe: one streaming pass over the probe rows that keeps the rows
// whose key may be in the table (and every row with the empty-marker key),
// appended with their row-ids through a per-warp stage, one atomic per flush.
__global__ void __launch_bounds__(PF_TPB) join_prefilter_kernel(const int64_t* keys, const uint32_t* rowids,
                                                                uint64_t n, const uint32_t* bloom, uint64_t bmask,
                                                                ProbeCtl* ctl, int64_t* out_keys,
                                                                uint32_t* out_rowids) {
    if (!ctl->active) return;
    __shared__ int64_t sk[PF_TPB / 32][PF_WCAP];
    __shared__ uint32_t sr[PF_TPB / 32][PF_WCAP];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    int64_t* wk = sk[warp];
    uint32_t* wr = sr[warp];
    unsigned cnt = 0;
    auto flush = [&]() {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0 && cnt) base = atomicAdd(&ctl->count, static_cast<unsigned long long>(cnt));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (unsigned i = lane; i < cnt; i += 32) {
            out_keys[base + i] = wk[i];
            out_rowids[base + i] = wr[i];
        }
        __syncwarp();
        cnt = 0;
    };
    constexpr uint64_t G = 32ull * PF_PER;
    const uint64_t groups = (n + G - 1) / G;
    const uint64_t nw = static_cast<uint64_t>(gridDim.x) * (PF_TPB / 32);
    for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * (PF_TPB / 32) + warp; g < groups; g += nw) {
        uint64_t key[PF_PER];
        bool keep[PF_PER];
#pragma unroll
        for (int j = 0; j < PF_PER; ++j) {
            const uint64_t i = g * G + static_cast<uint64_t>(j) * 32 + lane;
            key[j] = i < n ? ld_stream_u64(keys + i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < PF_PER; ++j) {
            const uint64_t i = g * G + static_cast<uint64_t>(j) * 32 + lane;
            const bool maybe = bloom_maybe(bloom, bmask, key[j]);
            keep[j] = i < n && (key[j] == JN_EMPTY || maybe);
        }
#pragma unroll
        for (int j = 0; j < PF_PER; ++j) {
            const uint64_t i = g * G + static_cast<uint64_t>(j) * 32 + lane;
            const unsigned b = __ballot_sync(0xFFFFFFFFu, keep[j]);
            if (cnt + 32 > PF_WCAP) flush();
            if (keep[j]) {
                const unsigned pos = cnt + __popc(b & ((1u << lane) - 1u));
                wk[pos] = static_cast<int64_t>(key[j]);
                wr[pos] = rowids ? ld_stream_u32(rowids + i) : static_cast<uint32_t>(i);
            }
            cnt += __popc(b);
        }
    }
    flush();
}

// ---- partitioned probe ------------------------------------------------------

constexpr int JQ_TPB = 256;
constexpr int JQ_PER = 8;                      // probe rows per thread per tile
constexpr int JQ_TILE = JQ_TPB * JQ_PER;       // rows per tile
constexpr int JQ_PMAX = 256;                   // most partitions
constexpr int JQ_CTAS_PER_SM = 4;              // grid of the two partition passes
static_assert(JQ_PMAX <= JQ_TPB, "one scan slot per partition");

struct PartArgs {
    const int64_t* keys;
    const uint32_t* rowids;                    // NULL => index
    uint64_t n;
    uint64_t mask;                             // buckets - 1
    int shift;                                 // partition = home bucket >> shift
    int parts;
    unsigned long long* cnt;                   // [gridDim.x][parts] rows per CTA and partition
    unsigned long long* pstart;                // [parts + 1] partition offsets (written by CTA 0)
    int64_t* out_keys;
    uint32_t* out_rowids;
    const ProbeCtl* pf;                        // non-NULL: the device-side plan (pre-probe, direct)
    const int64_t* pf_keys;                    // the pre-probe's surviving rows, used when pf->active
    const uint32_t* pf_rowids;
};

// The rows a partition pass reads: the probe's input, or the rows the Bloom
// pre-probe kept (decided on the device by the stage before).
__device__ __forceinline__ PartArgs part_source(const PartArgs& in) {
    PartArgs a = in;
    if (a.pf && a.pf->active) {
        a.keys = a.pf_keys;
        a.rowids = a.pf_rowids;
        a.n = a.pf->count;
    }
    return a;
}

__device__ __forceinline__ unsigned part_of(uint64_t key, const PartArgs& a) {
    return static_cast<unsigned>((fmix64(key) & a.mask) >> a.shift);
}

// Pass 1: rows of each partition in the tiles of this CTA (tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...).
__global__ void __launch_bounds__(JQ_TPB) join_part_count_kernel(PartArgs args) {
    if (args.pf && args.pf->direct) return;
    const PartArgs a = part_source(args);
    __shared__ unsigned h[JQ_PMAX];
    for (int p = threadIdx.x; p < a.parts; p += JQ_TPB) h[p] = 0;
    __syncthreads();
    for (uint64_t t0 = static_cast<uint64_t>(blockIdx.x) * JQ_TILE; t0 < a.n;
         t0 += static_cast<uint64_t>(gridDim.x) * JQ_TILE) {
        uint64_t k[JQ_PER];
#pragma unroll
        for (int j = 0; j < JQ_PER; ++j) {
            const uint64_t idx = t0 + static_cast<uint64_t>(j) * JQ_TPB + threadIdx.x;
            k[j] = idx < a.n ? ld_stream_u64(a.keys + idx) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < JQ_PER; ++j) {
            const uint64_t idx = t0 + static_cast<uint64_t>(j) * JQ_TPB + threadIdx.x;
            if (idx < a.n) atomicAdd(&h[part_of(k[j], a)], 1u);
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < a.parts; p += JQ_TPB)
        a.cnt[static_cast<uint64_t>(blockIdx.x) * a.parts + p] = h[p];
}

// Pass 2: the same tiles again; each row goes to its partition at this CTA's
// running offset (partition start + rows of that partition in lower CTAs +
// rows already placed), reordered in shared memory so the writes of a
// partition's run are contiguous.  The keys of the CTA's next tile are loaded
// while the current one is reordered.  Three CTA barriers per tile: the
// per-tile counts alternate between two arrays (the next tile's is zeroed
// while this one is scanned), one warp scans them, and the next tile cannot
// overwrite the reorder buffer before every thread has passed its first
// barrier, which it reaches only after writing this tile out.
__global__ void __launch_bounds__(JQ_TPB) join_part_scatter_kernel(PartArgs args) {
    if (args.pf && args.pf->direct) return;
    const PartArgs a = part_source(args);
    __shared__ unsigned h[2][JQ_PMAX];
    __shared__ unsigned off[JQ_PMAX];
    __shared__ unsigned long long base[JQ_PMAX];
    __shared__ unsigned long long tbase[JQ_PMAX];
    __shared__ unsigned long long wsum[JQ_TPB / 32];
    __shared__ unsigned long long total;
    __shared__ int64_t sk[JQ_TILE];
    __shared__ uint32_t sr[JQ_TILE];
    __shared__ uint8_t sp[JQ_TILE];
    const int p = threadIdx.x;
    const int P = a.parts;
    {
        unsigned long long below = 0, all = 0;
        if (p < P) {
            for (unsigned c = 0; c < gridDim.x; ++c) {
                const unsigned long long v = a.cnt[static_cast<uint64_t>(c) * P + p];
                all += v;
                if (c < blockIdx.x) below += v;
            }
        }
        const unsigned long long start = block_excl_scan<JQ_TPB>(all, wsum, &total);
        if (p < P) {
            base[p] = start + below;
            h[0][p] = 0;
        }
        if (blockIdx.x == 0 && p < P) a.pstart[p] = start;
        if (blockIdx.x == 0 && p == 0) a.pstart[P] = total;
    }
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    const int PP = (P + 31) / 32;                      // partitions per lane of the scanning warp
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * JQ_TILE;
    uint64_t kc[JQ_PER];
    const uint64_t first = static_cast<uint64_t>(blockIdx.x) * JQ_TILE;
#pragma unroll
    for (int j = 0; j < JQ_PER; ++j) {
        const uint64_t idx = first + static_cast<uint64_t>(j) * JQ_TPB + threadIdx.x;
        kc[j] = idx < a.n ? ld_stream_u64(a.keys + idx) : 0ull;
    }
    int cur = 0;
    for (uint64_t t0 = first; t0 < a.n; t0 += stride, cur ^= 1) {
        uint64_t kn[JQ_PER];
#pragma unroll
        for (int j = 0; j < JQ_PER; ++j) {
            const uint64_t idx = t0 + stride + static_cast<uint64_t>(j) * JQ_TPB + threadIdx.x;
            kn[j] = idx < a.n ? ld_stream_u64(a.keys + idx) : 0ull;
        }
        unsigned* hc = h[cur];
        unsigned pr[JQ_PER];                   // partition | rank in the tile << 8
#pragma unroll
        for (int j = 0; j < JQ_PER; ++j) {
            const uint64_t idx = t0 + static_cast<uint64_t>(j) * JQ_TPB + threadIdx.x;
            const unsigned q = part_of(kc[j], a);
            pr[j] = idx < a.n ? (q | (atomicAdd(&hc[q], 1u) << 8)) : 0u;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // the tile's run starts (exclusive scan of its counts), the
            // partitions' output positions, and the other count array zeroed
            unsigned run = 0;
            for (int i = 0; i < PP; ++i) {
                const int q = static_cast<int>(lane) * PP + i;
                if (q < P) run += hc[q];
            }
            unsigned incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= static_cast<unsigned>(o)) incl += v;
            }
            unsigned at = incl - run;
            for (int i = 0; i < PP; ++i) {
                const int q = static_cast<int>(lane) * PP + i;
                if (q < P) {
                    const unsigned c = hc[q];
                    off[q] = at;
                    tbase[q] = base[q];
                    base[q] += c;
                    h[cur ^ 1][q] = 0;
                    at += c;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < JQ_PER; ++j) {
            const uint64_t idx = t0 + static_cast<uint64_t>(j) * JQ_TPB + threadIdx.x;
            if (idx < a.n) {
                const unsigned q = pr[j] & 0xFFu;
                const unsigned pos = off[q] + (pr[j] >> 8);
                sk[pos] = static_cast<int64_t>(kc[j]);
                sr[pos] = a.rowids ? ld_stream_u32(a.rowids + idx) : static_cast<uint32_t>(idx);
                sp[pos] = static_cast<uint8_t>(q);
            }
        }
        __syncthreads();
        const unsigned len = static_cast<unsigned>(min(static_cast<uint64_t>(JQ_TILE), a.n - t0));
        for (unsigned i = threadIdx.x; i < len; i += JQ_TPB) {
            const unsigned q = sp[i];
            const unsigned long long dst = tbase[q] + (i - off[q]);
            a.out_keys[dst] = sk[i];
            a.out_rowids[dst] = sr[i];
        }
#pragma unroll
        for (int j = 0; j < JQ_PER; ++j) kc[j] = kn[j];
    }
}

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <typename K>
bool probe_kernel_setup(K kernel, int* per_sm) {
    int per = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, JP_SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, JP_TPB, JP_SMEM) != cudaSuccess)
        return false;
    *per_sm = std::min(*per_sm, per);
    return true;
}

int probe_grid(int device) {
    static std::atomic<int> cached[64] = {};
    if (device < 0 || device >= 64) return 0;
    if (const int c = cached[device].load()) return c;
    int sms = 0, per = 1 << 20;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (!probe_kernel_setup(join_probe_kernel<false>, &per) || !probe_kernel_setup(join_probe_kernel<true>, &per))
        return 0;
    cached[device].store(sms * std::max(1, per));
    return cached[device].load();
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Grid of the two partition passes.  Both take the same one (the scatter
// reads the count pass's per-CTA counts), at most JQ_CTAS_PER_SM per SM and no
// more than the heavier scatter kernel keeps resident: every CTA owns a fixed
// set of tiles, so CTAs beyond one wave would run their whole share late.
int part_grid(int device, int sms) {
    static std::atomic<int> cached[64] = {};
    if (device < 0 || device >= 64) return 0;
    if (const int c = cached[device].load()) return c;
    int per_s = 0, per_c = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_s, join_part_scatter_kernel, JQ_TPB, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_c, join_part_count_kernel, JQ_TPB, 0) != cudaSuccess)
        return 0;
    cached[device].store(sms * std::max(1, std::min(JQ_CTAS_PER_SM, std::min(per_s, per_c))));
    return cached[device].load();
}

}  // namespace

// Partitions the probe of `n` rows against `t` uses (1 = direct probe).
int probe_parts(const olap_ctx* ctx, const olap_join_table* t, uint64_t n) {
    const int opt = ctx->opts.join_partitions;
    uint64_t parts = 1;
    if (opt >= 2) {
        parts = static_cast<uint64_t>(opt);
    } else if (opt == 0) {
        const uint64_t tb = t->n_buckets * 32;
        const uint64_t l2 = ctx->l2_bytes ? ctx->l2_bytes : (64ull << 20);
        // worth it when the table is well above L2 and the probe side reads
        // at least a quarter as many buckets as the table has
        if (tb > l2 / 2 && n >= t->n_buckets / 4) parts = next_pow2((tb + l2 / 4 - 1) / (l2 / 4));
    }
    parts = std::min<uint64_t>(parts, static_cast<uint64_t>(JQ_PMAX));
    parts = std::min<uint64_t>(parts, t->n_buckets);
    return static_cast<int>(std::max<uint64_t>(parts, 1));
}

// Whether a probe of n rows against t runs the Bloom pre-probe stage (its
// sample still decides on the device whether rows are dropped).
bool probe_prefilter(const olap_ctx* ctx, const olap_join_table* t, uint64_t n) {
    if (!t->bloom || n == 0) return false;
    const int opt = ctx->opts.join_prefilter;
    return opt == OLAP_PREFILTER_ON || (opt == OLAP_PREFILTER_AUTO && n >= PF_MIN_N);
}

// Partition scratch: [partitioned keys | row-ids | count matrix | partition
// starts]; then, with the pre-probe, [kept keys | kept row-ids].  The probe's
// device-side plan lives in the context's small device area.
size_t probe_part_bytes(const olap_ctx* ctx, uint64_t n, int parts) {
    if (parts <= 1) return 0;
    // room for the largest grid the partition passes can take
    const uint64_t grid = static_cast<uint64_t>(ctx->sm_count) * JQ_CTAS_PER_SM;
    return align256(n * 8) + align256(n * 4) + align256(grid * parts * 8) + align256((parts + 1) * 8);
}

size_t probe_scratch_bytes(const olap_ctx* ctx, const olap_join_table* t, uint64_t n) {
    const size_t pb = probe_part_bytes(ctx, n, probe_parts(ctx, t, n));
    if (!probe_prefilter(ctx, t, n)) return pb;
    return pb + align256(n * 8) + align256(n * 4);
}

}  // namespace olap


using namespace olap;

namespace {

olap_status probe_enqueue(olap_ctx* ctx, const olap_join_table* t, const int64_t* d_keys, const uint32_t* d_rowids,
                          uint64_t n, olap_pair* d_out, uint64_t capacity, uint64_t* d_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "probe count reset");
    if (n == 0) {
        ctx->last_probe_parts = 1;
        ctx->last_probe_n = 0;
        ctx->last_probe_pf = nullptr;
        return OLAP_OK;
    }
    const int grid = probe_grid(ctx->device);
    if (grid <= 0) return fail(ctx, OLAP_E_CUDA, "probe kernel occupancy query failed");
    ProbeArgs a;
    a.keys = d_keys;
    a.rowids = d_rowids;
    a.n = n;
    a.slots = t->slots;
    a.mask = t->n_buckets - 1;
    a.side = t->side;
    a.n_side = t->n_side;
    a.out = reinterpret_cast<uint2*>(d_out);
    a.cap = capacity;
    a.count = reinterpret_cast<unsigned long long*>(d_count);
    const int parts = probe_parts(ctx, t, n);
    const bool pre = probe_prefilter(ctx, t, n);
    // the sample may still turn an automatically partitioned probe direct
    const bool skew_check = parts > 1 && ctx->opts.join_partitions == 0;
    PartArgs q{};
    unsigned qgrid = 0;
    ProbeCtl* pf = nullptr;
    int64_t* pf_keys = nullptr;
    uint32_t* pf_rowids = nullptr;
    if (parts > 1 || pre) {
        olap_status st = ensure_part(ctx, probe_scratch_bytes(ctx, t, n));
        if (st != OLAP_OK) return st;
    }
    if (pre || skew_check) pf = reinterpret_cast<ProbeCtl*>(static_cast<unsigned char*>(ctx->aux) + 1024);
    if (pre) {
        unsigned char* m = static_cast<unsigned char*>(ctx->part) + probe_part_bytes(ctx, n, parts);
        pf_keys = reinterpret_cast<int64_t*>(m);
        pf_rowids = reinterpret_cast<uint32_t*>(m + align256(n * 8));
        if (m + align256(n * 8) + align256(n * 4) > static_cast<unsigned char*>(ctx->part) + ctx->part_bytes)
            return fail(ctx, OLAP_E_INVALID, "probe pre-filter scratch too small");
    }
    if (parts > 1) {
        unsigned char* m = static_cast<unsigned char*>(ctx->part);
        qgrid = static_cast<unsigned>(part_grid(ctx->device, ctx->sm_count));
        if (qgrid == 0) return fail(ctx, OLAP_E_CUDA, "partition kernel occupancy query failed");
        q.keys = d_keys;
        q.rowids = d_rowids;
        q.n = n;
        q.mask = a.mask;
        q.shift = 0;
        while ((t->n_buckets >> q.shift) > static_cast<uint64_t>(parts)) ++q.shift;
        q.parts = parts;
        q.out_keys = reinterpret_cast<int64_t*>(m);
        q.out_rowids = reinterpret_cast<uint32_t*>(m + align256(n * 8));
        q.cnt = reinterpret_cast<unsigned long long*>(m + align256(n * 8) + align256(n * 4));
        q.pstart = q.cnt + static_cast<uint64_t>(qgrid) * parts;
        if (q.pstart + parts + 1 > reinterpret_cast<unsigned long long*>(m + ctx->part_bytes))
            return fail(ctx, OLAP_E_INVALID, "probe partition scratch too small");
        q.pf = pf;
        q.pf_keys = pf_keys;
        q.pf_rowids = pf_rowids;
    }
    ctx->last_probe_parts = parts;
    ctx->last_probe_n = n;
    ctx->last_probe_pf = pf;
    ctx->probe_timed = ctx->time_kernels;
    if (ctx->time_kernels && (e = cudaEventRecord(ctx->kev[4], s)) != cudaSuccess)
        return cuda_fail(ctx, e, "timing event");
    // the row queue's counter, in the context's small device area
    unsigned long long* next_row = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(ctx->aux) + 256);
    if ((e = cudaMemsetAsync(next_row, 0, sizeof(unsigned long long), s)) != cudaSuccess)
        return cuda_fail(ctx, e, "probe queue reset");
    ProbeArgs pa = a;
    const uint64_t bmask = pre ? t->bloom_blocks - 1 : 0;
    if (pf) {
        const int pf_mode = pre ? (ctx->opts.join_prefilter == OLAP_PREFILTER_ON ? 2 : 1) : 0;
        const int skew_l1 = ctx->opts.join_bucket_loads == OLAP_LOADS_AUTO ? 1 : 0;
        PlanArgs pl;
        pl.keys = d_keys;
        pl.rowids = d_rowids;
        pl.n = n;
        pl.bloom = pre ? t->bloom : nullptr;
        pl.bmask = bmask;
        pl.pf_mode = pf_mode;
        pl.skew_check = skew_check ? 1 : 0;
        pl.partitioned = parts > 1 ? 1 : 0;
        pl.skew_l1 = skew_l1;
        pl.pf_keys = pf_keys;
        pl.pf_rowids = pf_rowids;
        pl.sample = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ctx->aux) + 16384);
        pl.counters = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(ctx->aux) + 1536);
        pl.ctl = pf;
        join_probe_plan_kernel<<<PLAN_CTAS, PF_TPB, 0, s>>>(pl);
    }
    if (pre)
        join_prefilter_kernel<<<ctx->sm_count * 4, PF_TPB, 0, s>>>(d_keys, d_rowids, n, t->bloom, bmask, pf,
                                                                   pf_keys, pf_rowids);
    if (parts > 1) {
        join_part_count_kernel<<<qgrid, JQ_TPB, 0, s>>>(q);
        join_part_scatter_kernel<<<qgrid, JQ_TPB, 0, s>>>(q);
        pa.keys = q.out_keys;
        pa.rowids = q.out_rowids;
    }
    if (ctx->opts.join_bucket_loads == OLAP_LOADS_L1)
        join_probe_kernel<false><<<grid, JP_TPB, JP_SMEM, s>>>(pa, next_row, pf);
    else
        join_probe_kernel<true><<<grid, JP_TPB, JP_SMEM, s>>>(pa, next_row, pf);
    e = cudaGetLastError();
    // [plan,] [filter,] [count, scatter,] probe
    if (e == cudaSuccess) ctx->launches += (pf ? 1 : 0) + (pre ? 1 : 0) + (parts > 1 ? 2 : 0) + 1;
    if (e == cudaSuccess && ctx->time_kernels) e = cudaEventRecord(ctx->kev[5], s);
    return e == cudaSuccess ? OLAP_OK : cuda_fail(ctx, e, "probe launch");
}

olap_status check_join_table(olap_ctx* ctx, const olap_join_table* t) {
    if (!t || !t->slots) return fail(ctx, OLAP_E_INVALID, "join table is NULL or freed");
    if (t->device != ctx->device) return fail(ctx, OLAP_E_INVALID, "join table lives on another device");
    return OLAP_OK;
}

}  // namespace

extern "C" {

olap_status olap_join_build(olap_ctx* ctx, const int64_t* keys, const uint32_t* rowids, olap_mem where, uint64_t n,
                            double load_factor, olap_join_table** out) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!out) return fail(ctx, OLAP_E_INVALID, "out is NULL");
    *out = nullptr;
    if (where < OLAP_MEM_HOST || where > OLAP_MEM_DEVICE) return fail(ctx, OLAP_E_INVALID, "bad memory kind");
    if (n && !keys) return fail(ctx, OLAP_E_INVALID, "keys is NULL");
    if (!rowids && n > (1ull << 32)) return fail(ctx, OLAP_E_INVALID, "implicit row-ids need n <= 2^32");
    if (reinterpret_cast<uintptr_t>(keys) % 8) return fail(ctx, OLAP_E_INVALID, "keys misaligned");
    double load = load_factor > 0.0 ? load_factor : (ctx->opts.load_factor > 0.0 ? ctx->opts.load_factor : 0.5);
    if (!(load > 0.0 && load <= 0.9)) return fail(ctx, OLAP_E_INVALID, "load factor must be in (0, 0.9]");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");

    const uint64_t want_slots = static_cast<uint64_t>(static_cast<double>(n) / load) + 2;
    const uint64_t buckets = next_pow2((want_slots + 1) / 2);
    if (buckets > (1ull << 32)) return fail(ctx, OLAP_E_NOMEM, "join table: more than 2^32 buckets");
    const size_t slot_bytes = buckets * 32;
    // Bloom filter for the pre-probe: about 16 bits per build row, for tables
    // well above L2 (automatic) or every table with rows (forced on).
    const uint64_t l2 = ctx->l2_bytes ? ctx->l2_bytes : (64ull << 20);
    const bool with_bloom = n && (ctx->opts.join_prefilter == OLAP_PREFILTER_ON ||
                                  (ctx->opts.join_prefilter == OLAP_PREFILTER_AUTO && slot_bytes > l2 / 2));
    const uint64_t bloom_blocks = with_bloom ? next_pow2((n + 15) / 16) : 0;
    const size_t bytes = slot_bytes + 256 + bloom_blocks * 32;
    if (!within_budget(ctx, bytes)) return fail(ctx, OLAP_E_NOMEM, "join table: device memory budget exceeded");

    // Key-only input: build keys (and row-ids) to the device.
    const int64_t* dk = keys;
    const uint32_t* dr = rowids;
    if (where != OLAP_MEM_DEVICE && n) {
        const size_t kb = (n * 8 + 255) & ~static_cast<size_t>(255);
        olap_status st = ensure_dev_in(ctx, kb + (rowids ? n * 4 : 0));
        if (st != OLAP_OK) return st;
        st = copy_h2d(ctx, ctx->dev_in, keys, n * 8, where);
        if (st != OLAP_OK) return st;
        dk = static_cast<const int64_t*>(ctx->dev_in);
        if (rowids) {
            dr = reinterpret_cast<const uint32_t*>(static_cast<unsigned char*>(ctx->dev_in) + kb);
            st = copy_h2d(ctx, const_cast<uint32_t*>(dr), rowids, n * 4, where);
            if (st != OLAP_OK) return st;
        }
    }

    olap_join_table* t = new olap_join_table();
    t->device = ctx->device;
    t->n_buckets = buckets;
    t->n_build = n;
    t->load = load;
    void* mem = nullptr;
    e = cudaMalloc(&mem, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete t;
        return cuda_fail(ctx, e, "join table allocation");
    }
    t->slots = static_cast<ulonglong2*>(mem);
    t->bytes = bytes;
    JoinCtl* jc = reinterpret_cast<JoinCtl*>(static_cast<unsigned char*>(mem) + slot_bytes);
    auto bail = [&](olap_status st) {
        cudaFree(mem);
        delete t;
        return st;
    };
    if (bloom_blocks) {
        t->bloom = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(mem) + slot_bytes + 256);
        t->bloom_blocks = bloom_blocks;
    }
    e = cudaMemsetAsync(mem, 0xFF, slot_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(jc, 0, sizeof(JoinCtl), ctx->stream);
    if (e == cudaSuccess && bloom_blocks) e = cudaMemsetAsync(t->bloom, 0, bloom_blocks * 32, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "join table init"));
    if (n) {
        const int grid = ctx->sm_count * 8;
        join_build_kernel<<<grid, JB_TPB, 0, ctx->stream>>>(dk, dr, n, t->slots, buckets - 1, jc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "build launch"));
        join_chain_kernel<<<grid, JB_TPB, 0, ctx->stream>>>(t->slots, buckets - 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "build launch"));
        ctx->launches += 2;
        if (bloom_blocks) {
            join_bloom_kernel<<<grid, JB_TPB, 0, ctx->stream>>>(dk, n, t->bloom, bloom_blocks - 1);
            e = cudaGetLastError();
            if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "bloom launch"));
            ctx->launches += 1;
        }
    }
    JoinCtl hc;
    e = cudaMemcpyAsync(&hc, jc, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "join build"));
    if (hc.err) return bail(fail(ctx, static_cast<olap_status>(hc.err), "join build: table full"));
    if (hc.side_count) {
        e = cudaMalloc(reinterpret_cast<void**>(&t->side), hc.side_count * 4);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bail(cuda_fail(ctx, e, "join side list allocation"));
        }
        join_side_kernel<<<ctx->sm_count * 4, JB_TPB, 0, ctx->stream>>>(dk, dr, n, t->side, jc);
        e = cudaGetLastError();
        if (e == cudaSuccess) ctx->launches += 1;
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            cudaFree(t->side);
            return bail(cuda_fail(ctx, e, "join side list"));
        }
        t->n_side = hc.side_count;
        t->bytes += hc.side_count * 4;
    }
    ctx->table_bytes += t->bytes;
    ctx->tables.insert(t);
    t->owner = ctx;
    *out = t;
    return OLAP_OK;
}

olap_status olap_join_probe_async(olap_ctx* ctx, const olap_join_table* table, const int64_t* d_keys,
                                  const uint32_t* d_rowids, uint64_t n, olap_pair* d_out, uint64_t capacity,
                                  uint64_t* d_count, void* stream) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    olap_status st = check_join_table(ctx, table);
    if (st != OLAP_OK) return st;
    if (!d_count) return fail(ctx, OLAP_E_INVALID, "d_count is NULL");
    if (n && !d_keys) return fail(ctx, OLAP_E_INVALID, "keys is NULL");
    if (capacity && !d_out) return fail(ctx, OLAP_E_INVALID, "out is NULL");
    if (!d_rowids && n > (1ull << 32)) return fail(ctx, OLAP_E_INVALID, "implicit row-ids need n <= 2^32");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    return probe_enqueue(ctx, table, d_keys, d_rowids, n, d_out, capacity, d_count, s);
}

olap_status olap_join_probe(olap_ctx* ctx, const olap_join_table* table, const int64_t* keys,
                            const uint32_t* rowids, olap_mem where, uint64_t n, olap_pair* out, olap_mem out_where,
                            uint64_t capacity, uint64_t* out_count) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!out_count) return fail(ctx, OLAP_E_INVALID, "out_count is NULL");
    *out_count = 0;
    olap_status st = check_join_table(ctx, table);
    if (st != OLAP_OK) return st;
    if (where < OLAP_MEM_HOST || where > OLAP_MEM_DEVICE || out_where < OLAP_MEM_HOST ||
        out_where > OLAP_MEM_DEVICE)
        return fail(ctx, OLAP_E_INVALID, "bad memory kind");
    if (n && !keys) return fail(ctx, OLAP_E_INVALID, "keys is NULL");
    if (capacity && !out) return fail(ctx, OLAP_E_INVALID, "out is NULL");
    if (!rowids && n > (1ull << 32)) return fail(ctx, OLAP_E_INVALID, "implicit row-ids need n <= 2^32");
    if (reinterpret_cast<uintptr_t>(keys) % 8) return fail(ctx, OLAP_E_INVALID, "keys misaligned");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");

    const int64_t* dk = keys;
    const uint32_t* dr = rowids;
    if (where != OLAP_MEM_DEVICE && n) {
        const size_t kb = (n * 8 + 255) & ~static_cast<size_t>(255);
        st = ensure_dev_in(ctx, kb + (rowids ? n * 4 : 0));
        if (st != OLAP_OK) return st;
        st = copy_h2d(ctx, ctx->dev_in, keys, n * 8, where);
        if (st != OLAP_OK) return st;
        dk = static_cast<const int64_t*>(ctx->dev_in);
        if (rowids) {
            dr = reinterpret_cast<const uint32_t*>(static_cast<unsigned char*>(ctx->dev_in) + kb);
            st = copy_h2d(ctx, const_cast<uint32_t*>(dr), rowids, n * 4, where);
            if (st != OLAP_OK) return st;
        }
    }
    olap_pair* dout = out;
    // Device count word: a small slot at the end of the output staging area
    // (host outputs) or of the context scratch (device outputs).
    uint64_t* dcount = nullptr;
    if (out_where != OLAP_MEM_DEVICE) {
        const size_t ob = (capacity * 8 + 255) & ~static_cast<size_t>(255);
        st = ensure_dev_out(ctx, ob + 256);
        if (st != OLAP_OK) return st;
        dout = static_cast<olap_pair*>(ctx->dev_out);
        dcount = reinterpret_cast<uint64_t*>(static_cast<unsigned char*>(ctx->dev_out) + ob);
    } else {
        dcount = static_cast<uint64_t*>(ctx->aux);
    }
    st = probe_enqueue(ctx, table, dk, dr, n, dout, capacity, dcount, ctx->stream);
    if (st != OLAP_OK) return st;
    uint64_t cnt = 0;
    e = cudaMemcpyAsync(ctx->host_status + 8, dcount, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "join probe");
    std::memcpy(&cnt, ctx->host_status + 8, sizeof(cnt));
    *out_count = cnt;
    if (cnt > capacity) return fail(ctx, OLAP_E_OVERFLOW, "join probe: output capacity too small");
    if (out_where != OLAP_MEM_DEVICE && cnt) {
        st = copy_d2h(ctx, out, dout, cnt * 8, out_where);
        if (st != OLAP_OK) return st;
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "join result copy");
    }
    return OLAP_OK;
}

olap_status olap_join_probe_partitions(olap_ctx* ctx, const olap_join_table* table, uint64_t n, int* parts) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!parts) return fail(ctx, OLAP_E_INVALID, "parts is NULL");
    olap_status st = check_join_table(ctx, table);
    if (st != OLAP_OK) return st;
    *parts = probe_parts(ctx, table, n);
    return OLAP_OK;
}

olap_status olap_join_probe_info_last(olap_ctx* ctx, int* parts, int* prefiltered, uint64_t* rows_probed) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!parts || !prefiltered || !rows_probed) return fail(ctx, OLAP_E_INVALID, "NULL output");
    if (ctx->last_probe_parts == 0) return fail(ctx, OLAP_E_INVALID, "no probe has run on this context");
    *parts = ctx->last_probe_parts;
    *prefiltered = 0;
    *rows_probed = ctx->last_probe_n;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "probe info");
    if (ctx->last_probe_pf) {
        ProbeCtl c;
        e = cudaMemcpy(&c, ctx->last_probe_pf, sizeof(c), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "probe info");
        if (c.active) {
            *prefiltered = 1;
            *rows_probed = c.count;
        }
        if (c.direct) *parts = 1;
    }
    return OLAP_OK;
}

olap_status olap_join_table_info(const olap_join_table* t, uint64_t* n_build, uint64_t* n_buckets, uint64_t* n_side,
                                 uint64_t* bloom_bytes) {
    if (!t || !t->slots) return OLAP_E_INVALID;
    if (n_build) *n_build = t->n_build;
    if (n_buckets) *n_buckets = t->n_buckets;
    if (n_side) *n_side = t->n_side;
    if (bloom_bytes) *bloom_bytes = t->bloom_blocks * 32;
    return OLAP_OK;
}

void olap_join_free(olap_join_table* t) {
    if (!t) return;
    if (t->owner) {
        t->owner->table_bytes -= t->bytes;
        t->owner->tables.erase(t);
    }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(t->device);
    cudaDeviceSynchronize();
    if (t->slots) cudaFree(t->slots);
    if (t->side) cudaFree(t->side);
    t->slots = nullptr;
    t->side = nullptr;
    cudaSetDevice(cur);
    delete t;
}

}  // extern "C"

void detach_tables(olap_ctx* ctx) {
    for (olap_join_table* t : ctx->tables) t->owner = nullptr;
    ctx->tables.clear();
}
