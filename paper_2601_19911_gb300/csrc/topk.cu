// Top-K selection over key-only (key, row-id) columns: ORDER BY key LIMIT K
// (Sec. III-A, "partial selection (or radix-based selection)", returning the
// row pointers of the Top-K rows in order).
//
// Three launches on one stream:
//   0. topk_prepare_kernel zeroes the control block and, when N > 2^21 and K
//      is small against N, reads a stratified sample of 8192 keys (16 CTAs,
//      one key per thread) and finds the rank word of the sample's r-th best
//      entry by a radix select in the last CTA to finish; r is chosen so that,
//      with high probability, at least K keys but not many more fall at or
//      below it.
//   1. topk_filter_regs_kernel (default) or topk_filter_bulk_kernel (TMA
//      bulk copies into a shared-memory ring): the only full pass over the
//      keys, run only when there is a sample.  16-byte streaming loads, one
//      compare per key against the threshold in the key's own bit domain,
//      and every key that passes is appended (per-warp staging, one global
//      atomic per flush) to a candidate buffer with its row-id.
//   Phases 2-4 are one cooperative launch (topk_select_kernel) whose CTAs
//   meet at bounded grid barriers.  Its source is the candidate buffer when
//   the sample worked (at least K candidates, no overflow) and the full
//   input otherwise (no sample, or a misjudged one).
//   2. Refine: radix passes of 12-bit digits over the (key, row-id) composite
//      of the candidates (or the input): a shared-memory histogram with
//      __match_any_sync aggregation, merged into a global histogram; every
//      CTA then scans it and extends the same prefix, until the bucket that
//      holds the K-th entry has at most 4096 entries.
//   3. Split: entries below the prefix are selected; entries equal to it go
//      to a small buffer that one CTA sorts to take the remaining count.
//   4. Sort the K survivors by (rank word, row-id) -- in shared memory when
//      K <= 4096, else tile sorts plus merge-path rounds across the grid --
//      and write keys (original bits, by the inverse transform) and row-ids.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "block.cuh"
#include "topk.cuh"

namespace olap {

namespace {

struct Elem {
    uint64_t r;
    uint32_t rid;
};

// Rank word of a two-column key: c0's 32-bit rank above c1's.
__device__ __forceinline__ uint64_t pair_rank(uint32_t b0, uint32_t b1, const TopkArgs& a) {
    return rank_key(b0, a.kind, a.desc) | (rank_key(b1, a.kind2, a.desc2) >> 32);
}

__device__ __forceinline__ Elem load_input(const TopkArgs& a, uint64_t i) {
    Elem e;
    if (a.pair) {
        e.r = pair_rank(static_cast<const uint32_t*>(a.keys)[i], static_cast<const uint32_t*>(a.keys2)[i], a);
    } else {
        const uint64_t bits = a.w4 ? static_cast<uint64_t>(static_cast<const uint32_t*>(a.keys)[i])
                                   : static_cast<const uint64_t*>(a.keys)[i];
        e.r = rank_key(bits, a.kind, a.desc);
    }
    e.rid = a.rowids ? a.rowids[i] : static_cast<uint32_t>(i);
    return e;
}

__device__ __forceinline__ Elem load_src(const TopkArgs& a, bool cand, uint64_t i) {
    if (cand) return Elem{__ldcg(a.cand_r + i), __ldcg(a.cand_rid + i)};
    return load_input(a, i);
}

__device__ __forceinline__ void write_result(const TopkArgs& a, uint64_t i, uint64_t r, uint32_t rid) {
    if (a.pair) {
        static_cast<uint32_t*>(a.out_keys)[i] = static_cast<uint32_t>(unrank_key(r & 0xFFFFFFFF00000000ull, a.kind, a.desc));
        static_cast<uint32_t*>(a.out_keys2)[i] = static_cast<uint32_t>(unrank_key(r << 32, a.kind2, a.desc2));
    } else if (a.w4)
        static_cast<uint32_t*>(a.out_keys)[i] = static_cast<uint32_t>(unrank_key(r, a.kind, a.desc));
    else
        static_cast<uint64_t*>(a.out_keys)[i] = unrank_key(r, a.kind, a.desc);
    a.out_rowids[i] = rid;
}

// Prepare kernel: a threshold rank word for the streaming pass from a
// stratified sample of TK_SAMPLE keys (sample j is key (j * n) / TK_SAMPLE +
// (n / TK_SAMPLE) / 2).  The prepare CTAs load it together, one key per
// thread, into a.samples -- from one SM, 8192 scattered loads wait on each
// other's DRAM latency -- and the last CTA to finish runs this radix select
// with a.digit-bit digits on the sample held in registers; it stops as soon as
// the upper edge of the chosen bucket has between r and r + 8 samples at or
// below it (any such threshold serves), which for spread-out keys is after the
// first digit.
__device__ uint64_t sample_threshold(const TopkArgs& a, unsigned* sh, unsigned long long* sc) {
    uint64_t s[TK_SPT];
#pragma unroll
    for (int j = 0; j < TK_SPT; ++j) s[j] = __ldcg(a.samples + static_cast<uint64_t>(j) * TK_TPB + threadIdx.x);
    const int kb = a.w4 ? 32 : 64;
    const unsigned long long r = a.sample_rank;
    uint64_t prefix = 0;
    unsigned long long rem = r, cum = 0;
    for (int L = 0; L < kb; L += a.digit) {
        const int d = min(a.digit, kb - L);
        for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB) sh[b] = 0;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TK_SPT; ++j) {
            const bool match = (L == 0) || (((s[j] ^ prefix) >> (64 - L)) == 0);
            if (match) atomicAdd(&sh[static_cast<unsigned>((s[j] << L) >> (64 - d))], 1u);
        }
        __syncthreads();
        const Pick pk = pick_bucket<TK_TPB>(sh, rem, sc);
        prefix |= static_cast<uint64_t>(pk.b) << (64 - L - d);
        rem -= pk.below;
        cum += pk.below;
        if (cum + pk.in_b <= r + 8) return prefix | ((1ull << (64 - L - d)) - 1ull);
    }
    return prefix;
}

// Hits of the streaming pass are staged per warp in shared memory and
// flushed to the global candidate buffer WS_CAP at a time: one atomic on the
// global count per flush instead of one per warp-vector with a hit (a single
// global counter hit by every SM serialises in L2), and coalesced writes.
constexpr int WS_CAP = 256;
struct WarpStage {
    uint64_t* r;          // WS_CAP rank words (shared)
    uint32_t* idx;        // WS_CAP key indices (shared)
    unsigned count;       // entries held (the same in every lane)
};
constexpr int WS_BYTES = WS_CAP * 12;

__device__ __forceinline__ WarpStage warp_stage(unsigned char* base) {
    const unsigned w = threadIdx.x >> 5;
    unsigned char* p = base + static_cast<size_t>(w) * WS_BYTES;
    return WarpStage{reinterpret_cast<uint64_t*>(p), reinterpret_cast<uint32_t*>(p + WS_CAP * 8), 0u};
}

// The select's first radix pass, folded into the streaming filter (the
// register and two-column filters).  Every candidate already passes through
// a warp stage; as it leaves, its digit at the first bit where candidates can
// differ (just below the threshold's leading zeros, the select's first pass
// position) is counted in a CTA histogram in shared memory, which the CTA adds
// to the select's pass-0 histogram when it is done.  The select then starts
// at the bucket pick, one pass over the candidates and one grid barrier
// sooner.  (The pass's AND / OR fold, which lets a pass skip bits all its
// entries share, is left to the select's later passes: four 64-bit shared
// atomics per candidate slowed the streaming pass by 5-10 %.)
__shared__ unsigned g_fuse_hist[TK_BINS];

// Bit position and width of the fused digit (those of the select's first pass).
struct FuseDigit {
    int L, d, kb;
};
__device__ __forceinline__ FuseDigit fuse_digit(const TopkArgs& a, uint64_t t) {
    FuseDigit f;
    f.kb = a.w4 ? 32 : 64;
    const int lz = __clzll(static_cast<long long>(t));
    f.L = lz < f.kb ? lz : f.kb;
    f.d = min(a.digit, f.kb + 32 - f.L);
    return f;
}

template <int TPB>
__device__ __forceinline__ void fuse_init() {
    for (int b = threadIdx.x; b < TK_BINS; b += TPB) g_fuse_hist[b] = 0;
    __syncthreads();
}

__device__ __forceinline__ void fuse_add(const FuseDigit& f, uint64_t r, uint32_t rid) {
    uint64_t w0, w1;
    comp_words(r, rid, f.kb, w0, w1);
    atomicAdd(&g_fuse_hist[comp_digit(w0, w1, f.L, f.d)], 1u);
}

// Whole CTA, after its last candidate: add the CTA's counts to the pass-0
// histogram (non-zero bins only).
template <int TPB>
__device__ __forceinline__ void fuse_merge(const TopkArgs& a) {
    __syncthreads();
    for (int b = threadIdx.x; b < TK_BINS; b += TPB)
        if (g_fuse_hist[b]) atomicAdd(&a.ghist[b], g_fuse_hist[b]);
}

// Programmatic dependent launch.  The filter and the select are launched
// while the kernel before them in the stream is still running; they wait here
// until it has finished and its writes are visible (measured, 2^28 int64
// keys: 3 us less per call).  A kernel launched without the attribute passes
// straight through.
__device__ __forceinline__ void wait_prior_grid() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
// Lets the next kernel in the stream launch now (it still waits for this one
// to finish before it reads anything).
__device__ __forceinline__ void allow_next_grid() {
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

// Move the warp's staged hits to the candidate buffer (all 32 lanes call).
__device__ __forceinline__ void stage_flush_plain(const TopkArgs& a, WarpStage& ws) {
    if (ws.count == 0) return;
    __syncwarp();
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.ctl->cand_count, static_cast<unsigned long long>(ws.count));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (unsigned j = lane; j < ws.count; j += 32) {
        const unsigned long long pos = base + j;
        if (pos < a.cand_cap) {
            const uint32_t idx = ws.idx[j];
            a.cand_r[pos] = ws.r[j];
            a.cand_rid[pos] = a.rowids ? a.rowids[idx] : idx;
        }
    }
    __syncwarp();
    ws.count = 0;
}

// The same, also counting the hits for the fused first pass.  Kept out of
// line: it runs once per WS_CAP hits of a warp, and inlined into the
// filter's unrolled loop it would cost the loop registers (occupancy).
__device__ __forceinline__ void stage_flush_fused(const TopkArgs& a, const uint64_t* sr, const uint32_t* sidx,
                                               unsigned count) {
    __syncwarp();
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.ctl->cand_count, static_cast<unsigned long long>(count));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    const FuseDigit f = fuse_digit(a, __ldcg(&a.ctl->thresh));
    for (unsigned j = lane; j < count; j += 32) {
        const unsigned long long pos = base + j;
        const uint32_t idx = sidx[j];
        const uint64_t r = sr[j];
        const uint32_t rid = a.rowids ? a.rowids[idx] : idx;
        if (pos < a.cand_cap) {
            a.cand_r[pos] = r;
            a.cand_rid[pos] = rid;
        }
        fuse_add(f, r, rid);
    }
    __syncwarp();
}

template <bool FUSE = false>
__device__ __forceinline__ void stage_flush(const TopkArgs& a, WarpStage& ws) {
    if (!FUSE) {
        stage_flush_plain(a, ws);
        return;
    }
    if (ws.count == 0) return;
    stage_flush_fused(a, ws.r, ws.idx, ws.count);
    ws.count = 0;
}

// Test the VEC keys of one 16-byte vector (keys idx0 .. idx0 + VEC - 1)
// against the threshold and stage the hits.  Called by all 32 lanes of a
// warp together.
template <bool W4, bool FUSE = false>
__device__ __forceinline__ void filter_vector(const TopkArgs& a, const KeyLimit& lim, uint4 x, bool valid,
                                              uint64_t idx0, WarpStage& ws) {
    constexpr int VEC = W4 ? 4 : 2;
    bool any;
    if (W4) {
        any = pass32(x.x, lim) | pass32(x.y, lim) | pass32(x.z, lim) | pass32(x.w, lim);
    } else {
        any = pass64(static_cast<uint64_t>(x.x) | (static_cast<uint64_t>(x.y) << 32), lim) |
              pass64(static_cast<uint64_t>(x.z) | (static_cast<uint64_t>(x.w) << 32), lim);
    }
    if (!__any_sync(0xFFFFFFFFu, any && valid)) return;
    unsigned hit = 0;
    if (valid) {
        if (W4) {
            hit = (pass32(x.x, lim) ? 1u : 0u) | (pass32(x.y, lim) ? 2u : 0u) | (pass32(x.z, lim) ? 4u : 0u) |
                  (pass32(x.w, lim) ? 8u : 0u);
        } else {
            hit = (pass64(static_cast<uint64_t>(x.x) | (static_cast<uint64_t>(x.y) << 32), lim) ? 1u : 0u) |
                  (pass64(static_cast<uint64_t>(x.z) | (static_cast<uint64_t>(x.w) << 32), lim) ? 2u : 0u);
        }
    }
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    unsigned bal[VEC];
    unsigned total = 0;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        bal[e] = __ballot_sync(0xFFFFFFFFu, (hit >> e) & 1u);
        total += __popc(bal[e]);
    }
    if (ws.count + total > WS_CAP) stage_flush<FUSE>(a, ws);
    unsigned before = ws.count;
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        if ((hit >> e) & 1u) {
            const unsigned pos = before + __popc(bal[e] & lt);
            uint64_t r;
            if (W4) r = rank_key(w[e], a.kind, a.desc);
            else r = rank_key(static_cast<uint64_t>(w[2 * e]) | (static_cast<uint64_t>(w[2 * e + 1]) << 32), a.kind, a.desc);
            ws.r[pos] = r;
            ws.idx[pos] = static_cast<uint32_t>(idx0 + e);
        }
        before += __popc(bal[e]);
    }
    ws.count += total;
}

// The unaligned head [0, head) and ragged tail [tail0, n) of the keys: at
// most 2 * VEC - 2 keys, one per lane of warp 0 of CTA 0.
template <bool FUSE = false>
__device__ __forceinline__ void filter_ends(const TopkArgs& a, uint64_t t, uint64_t head, uint64_t tail0) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const uint64_t rest = head + (a.n - tail0);
    const uint64_t j = threadIdx.x;
    const bool valid = j < rest;
    uint64_t idx = 0, r = ~0ull;
    if (valid) {
        idx = j < head ? j : tail0 + (j - head);
        r = load_input(a, idx).r;
    }
    const bool hit = valid && r <= t;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
    if (!bal) return;
    unsigned long long base = 0;
    if (threadIdx.x == 0) base = atomicAdd(&a.ctl->cand_count, static_cast<unsigned long long>(__popc(bal)));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (hit) {
        const unsigned long long pos = base + __popc(bal & ((1u << threadIdx.x) - 1u));
        const uint32_t rid = a.rowids ? a.rowids[idx] : static_cast<uint32_t>(idx);
        if (pos < a.cand_cap) {
            a.cand_r[pos] = r;
            a.cand_rid[pos] = rid;
        }
        if (FUSE) fuse_add(fuse_digit(a, t), r, rid);
    }
}

// Phase 1: the single streaming pass.  Appends (rank word, row-id) of every
// key whose rank word is <= t; counts all of them.
template <bool W4, int TPB>
__device__ void filter_pass(const TopkArgs& a, uint64_t t, unsigned char* stage_smem) {
    constexpr int W = W4 ? 4 : 8;
    constexpr int VEC = 16 / W;
    const uint64_t n = a.n;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(a.keys);
    const uint64_t head0 = ((16 - (addr & 15)) & 15) / W;
    const uint64_t head = head0 < n ? head0 : n;
    const uint64_t nvec = (n - head) / VEC;
    const uint64_t tail0 = head + nvec * VEC;
    const unsigned char* vbase = static_cast<const unsigned char*>(a.keys) + head * W;
    const KeyLimit lim = key_limit(t, a.kind, a.desc);
    WarpStage ws = warp_stage(stage_smem);

    const uint64_t per_block = static_cast<uint64_t>(TPB) * TK_UNROLL;
    const uint64_t stride = per_block * gridDim.x;
    for (uint64_t bb = per_block * blockIdx.x; bb < nvec; bb += stride) {
        uint4 v[TK_UNROLL];
#pragma unroll
        for (int u = 0; u < TK_UNROLL; ++u) {
            const uint64_t vi = bb + static_cast<uint64_t>(u) * TPB + threadIdx.x;
            if (vi < nvec) v[u] = ld_stream_v4(vbase + vi * 16);
            else v[u] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        }
#pragma unroll
        for (int u = 0; u < TK_UNROLL; ++u) {
            const uint64_t vi = bb + static_cast<uint64_t>(u) * TPB + threadIdx.x;
            filter_vector<W4, true>(a, lim, v[u], vi < nvec, head + vi * VEC, ws);
        }
    }
    stage_flush<true>(a, ws);
    filter_ends<true>(a, t, head, tail0);
}

// The 32-bit order-preserving transform of one 4-byte key kind as two masks:
// rank = b ^ (sign-extended top bit of b & flip) ^ fixed.  float32 flips the
// magnitude of negatives and sets the sign bit of the others (IEEE
// totalOrder), int32 flips the sign bit, uint32 keeps the bits; DESC
// complements the result.  The same map as rank_key, without branches.
struct Rank32 {
    uint32_t flip, fixed;
};
__device__ __forceinline__ Rank32 rank32_of(int kind, bool desc) {
    Rank32 m;
    m.flip = kind == OLAP_KEY_F32 ? 0x7FFFFFFFu : 0u;
    m.fixed = (kind == OLAP_KEY_U32 ? 0u : 0x80000000u) ^ (desc ? 0xFFFFFFFFu : 0u);
    return m;
}
__device__ __forceinline__ uint32_t rank32(uint32_t b, Rank32 m) {
    return b ^ (static_cast<uint32_t>(static_cast<int32_t>(b) >> 31) & m.flip) ^ m.fixed;
}

// Stage the hits among the four rows of one 16-byte vector of each column.
__device__ __forceinline__ void filter_vector_pair(const TopkArgs& a, uint64_t t, Rank32 m0, Rank32 m1, uint4 x0,
                                                   uint4 x1, bool valid, uint64_t idx0, WarpStage& ws) {
    const uint32_t c0[4] = {x0.x, x0.y, x0.z, x0.w}, c1[4] = {x1.x, x1.y, x1.z, x1.w};
    uint64_t r[4];
    unsigned hit = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        r[e] = (static_cast<uint64_t>(rank32(c0[e], m0)) << 32) | rank32(c1[e], m1);
        hit |= (valid && r[e] <= t) ? (1u << e) : 0u;
    }
    if (!__any_sync(0xFFFFFFFFu, hit != 0)) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt = (1u << lane) - 1u;
    unsigned bal[4];
    unsigned total = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        bal[e] = __ballot_sync(0xFFFFFFFFu, (hit >> e) & 1u);
        total += __popc(bal[e]);
    }
    if (ws.count + total > WS_CAP) stage_flush<true>(a, ws);
    unsigned before = ws.count;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if ((hit >> e) & 1u) {
            const unsigned pos = before + __popc(bal[e] & lt);
            ws.r[pos] = r[e];
            ws.idx[pos] = static_cast<uint32_t>(idx0 + e);
        }
        before += __popc(bal[e]);
    }
    ws.count += total;
}

// Phase 1 for a two-column key: both columns streamed with 16-byte loads when
// they share their alignment (a scalar head and tail around the vectors),
// else row by row; every row whose composite rank word is <= t is appended.
constexpr int TK_PAIR_UNROLL = 2;          // vector pairs (32 bytes) in flight per thread

template <int TPB>
__device__ void filter_pass_pair(const TopkArgs& a, uint64_t t, unsigned char* stage_smem) {
    const uint64_t n = a.n;
    const Rank32 m0 = rank32_of(a.kind, a.desc), m1 = rank32_of(a.kind2, a.desc2);
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a.keys), a1 = reinterpret_cast<uintptr_t>(a.keys2);
    WarpStage ws = warp_stage(stage_smem);
    const unsigned lane = threadIdx.x & 31u;
    if (((a0 ^ a1) & 15) == 0) {
        const uint64_t head0 = ((16 - (a0 & 15)) & 15) / 4;
        const uint64_t head = head0 < n ? head0 : n;
        const uint64_t nvec = (n - head) / 4;
        const uint64_t tail0 = head + nvec * 4;
        const unsigned char* v0 = static_cast<const unsigned char*>(a.keys) + head * 4;
        const unsigned char* v1 = static_cast<const unsigned char*>(a.keys2) + head * 4;
        const uint64_t per_block = static_cast<uint64_t>(TPB) * TK_PAIR_UNROLL;
        const uint64_t stride = per_block * gridDim.x;
        for (uint64_t bb = per_block * blockIdx.x; bb < nvec; bb += stride) {
            uint4 x0[TK_PAIR_UNROLL], x1[TK_PAIR_UNROLL];
#pragma unroll
            for (int u = 0; u < TK_PAIR_UNROLL; ++u) {
                const uint64_t vi = bb + static_cast<uint64_t>(u) * TPB + threadIdx.x;
                if (vi < nvec) {
                    x0[u] = ld_stream_v4(v0 + vi * 16);
                    x1[u] = ld_stream_v4(v1 + vi * 16);
                } else {
                    x0[u] = x1[u] = make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < TK_PAIR_UNROLL; ++u) {
                const uint64_t vi = bb + static_cast<uint64_t>(u) * TPB + threadIdx.x;
                filter_vector_pair(a, t, m0, m1, x0[u], x1[u], vi < nvec, head + vi * 4, ws);
            }
        }
        stage_flush<true>(a, ws);
        filter_ends<true>(a, t, head, tail0);
        return;
    }
    const uint64_t stride = static_cast<uint64_t>(TPB) * gridDim.x;
    const uint64_t lt = (1u << lane) - 1u;
    for (uint64_t wb = static_cast<uint64_t>(blockIdx.x) * TPB + (threadIdx.x & ~31u); wb < n; wb += stride) {
        const uint64_t i = wb + lane;
        uint64_t r = ~0ull;
        if (i < n) r = pair_rank(static_cast<const uint32_t*>(a.keys)[i], static_cast<const uint32_t*>(a.keys2)[i], a);
        const bool hit = i < n && r <= t;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
        if (!bal) continue;
        if (ws.count + __popc(bal) > WS_CAP) stage_flush<true>(a, ws);
        if (hit) {
            const unsigned pos = ws.count + __popc(bal & static_cast<unsigned>(lt));
            ws.r[pos] = r;
            ws.idx[pos] = static_cast<uint32_t>(i);
        }
        ws.count += __popc(bal);
    }
    stage_flush<true>(a, ws);
}

// Issue the bulk copy of the tile at byte offset `off` of the key body into
// ring slot `s` (the last tile of the body may be short).
__device__ __forceinline__ void issue_tile(unsigned char* smem, uint64_t* full, const unsigned char* vbase,
                                           uint64_t body, uint64_t off, uint32_t s, uint32_t tile,
                                           uint64_t policy) {
    const uint64_t left = body - off;
    const uint32_t bytes = static_cast<uint32_t>(left < tile ? left : tile);
    mbar_arrive_expect_tx(&full[s], bytes);
    bulk_g2s(smem + static_cast<size_t>(s) * tile, vbase + off, bytes, &full[s], policy);
}

// Phase 1, bulk-copy flavour: each CTA streams its tiles (tile i of the
// grid-interleaved order) through a ring of `stages` shared-memory slots.
// Thread 0 issues cp.async.bulk copies; a slot's "full" mbarrier completes
// when its bytes land, and its "empty" mbarrier when every warp has read it,
// after which thread 0 refills it.  No CTA-wide barrier per tile.  Returns
// false if a copy never landed (bounded waits).
template <bool W4, int TPB>
__device__ bool filter_pass_bulk(const TopkArgs& a, uint64_t t, unsigned char* smem) {
    constexpr int W = W4 ? 4 : 8;
    constexpr int VEC = 16 / W;
    constexpr unsigned NWARPS = TPB / 32;
    const uint32_t tile = static_cast<uint32_t>(a.tile_bytes);
    const uint32_t stages = static_cast<uint32_t>(a.stages);
    const uint64_t n = a.n;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(a.keys);
    const uint64_t head0 = ((16 - (addr & 15)) & 15) / W;
    const uint64_t head = head0 < n ? head0 : n;
    const uint64_t nvec = (n - head) / VEC;
    const uint64_t tail0 = head + nvec * VEC;
    const unsigned char* vbase = static_cast<const unsigned char*>(a.keys) + head * W;
    const uint64_t body = nvec * 16;
    const uint64_t ntiles = (body + tile - 1) / tile;
    const uint64_t my_n = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const KeyLimit lim = key_limit(t, a.kind, a.desc);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(tile) * stages);
    uint64_t* empty = full + TK_MAX_STAGES;
    WarpStage ws = warp_stage(reinterpret_cast<unsigned char*>(empty + TK_MAX_STAGES));
    const uint64_t step = static_cast<uint64_t>(gridDim.x) * tile;       // bytes between my tiles

    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NWARPS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t policy = l2_evict_first_policy();
    uint64_t off = static_cast<uint64_t>(blockIdx.x) * tile;
    uint64_t issued = 0;                                   // tiles issued (thread 0)
    if (threadIdx.x == 0) {
        const uint32_t pre = static_cast<uint32_t>(my_n < stages ? my_n : stages);
        for (uint32_t s = 0; s < pre; ++s) issue_tile(smem, full, vbase, body, off + s * step, s, tile, policy);
        issued = pre;
    }
    const uint64_t refill = static_cast<uint64_t>(stages) * step;
    const unsigned lane = threadIdx.x & 31u;
    uint32_t s = 0, par = 0;
    bool ok = true;
    for (uint64_t i = 0; i < my_n; ++i) {
        if (!mbar_wait(&full[s], par)) {
            ok = false;
            break;
        }
        const uint64_t left = body - off;
        const uint32_t nv = static_cast<uint32_t>((left < tile ? left : tile) / 16);
        const unsigned char* st = smem + static_cast<size_t>(s) * tile;
        const uint64_t idx_base = head + (off / 16) * VEC;
        for (uint32_t vb = 0; vb < tile / 16; vb += TPB) {
            const uint32_t v = vb + threadIdx.x;
            const bool valid = v < nv;
            uint4 x = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
            if (valid) x = ld_shared_v4(st + v * 16);
            filter_vector<W4>(a, lim, x, valid, idx_base + static_cast<uint64_t>(v) * VEC, ws);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (threadIdx.x == 0 && i + stages < my_n) {
            if (!mbar_wait(&empty[s], par)) {
                ok = false;
                break;
            }
            fence_proxy_async_smem();
            issue_tile(smem, full, vbase, body, off + refill, s, tile, policy);
            ++issued;
        }
        off += step;
        if (++s == stages) {
            s = 0;
            par ^= 1u;
        }
    }
    stage_flush(a, ws);
    if (!__syncthreads_and(ok)) {
        // Let the copies this CTA issued land before leaving.  Only the last
        // `stages` issued tiles can still be in flight (every earlier fill of
        // a slot was consumed before the slot was refilled).
        if (threadIdx.x == 0) {
            const uint64_t first = issued > stages ? issued - stages : 0;
            for (uint64_t q = first; q < issued; ++q)
                mbar_wait(&full[q % stages], static_cast<uint32_t>((q / stages) & 1));
            atomicCAS(&a.ctl->err, 0, static_cast<int>(OLAP_E_TIMEOUT));
        }
        __syncthreads();
        return false;
    }
    filter_ends(a, t, head, tail0);
    return true;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One refine pass: histogram of digit [L, L+d) of the composites that match
// the prefix, merged into `gh`, and the AND / OR of those composites merged
// into `ao`.  `gz` and `az` (the buffers of the pass after next) are reset by
// CTA 0.
__device__ void hist_pass(const TopkArgs& a, bool cand, uint64_t src_n, uint64_t p0, uint64_t p1,
                          int L, int d, int kb, unsigned* gh, unsigned* gz, unsigned* sh, unsigned long long* ao,
                          unsigned long long* az) {
    for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB) sh[b] = 0;
    if (blockIdx.x == 0) {
        for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB) gz[b] = 0;
        if (threadIdx.x == 0) {
            az[0] = az[1] = ~0ull;
            az[2] = az[3] = 0ull;
        }
    }
    __syncthreads();
    uint64_t acc[4] = {~0ull, ~0ull, 0ull, 0ull};
    const uint64_t stride = static_cast<uint64_t>(TK_TPB) * gridDim.x;
    const unsigned lane = threadIdx.x & 31u;
    for (uint64_t wb = static_cast<uint64_t>(blockIdx.x) * TK_TPB + (threadIdx.x & ~31u); wb < src_n;
         wb += stride) {
        const uint64_t i = wb + lane;
        unsigned dig = 0xFFFFFFFFu;
        if (i < src_n) {
            const Elem e = load_src(a, cand, i);
            uint64_t w0, w1;
            comp_words(e.r, e.rid, kb, w0, w1);
            if (prefix_cmp(w0, w1, p0, p1, L) == 0) {
                dig = comp_digit(w0, w1, L, d);
                and_or(w0, w1, acc);
            }
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
        if (dig != 0xFFFFFFFFu && lane == static_cast<unsigned>(__ffs(peers) - 1))
            atomicAdd(&sh[dig], static_cast<unsigned>(__popc(peers)));
    }
    and_or_merge<TK_TPB>(acc, ao);
    for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB)
        if (sh[b]) atomicAdd(&gh[b], sh[b]);
}

// Split: entries below the prefix are selected (appended to out), entries
// equal to it go to the small buffer, or straight to out when all of them
// (or any `krem` identical ones) are taken.
// With FOLD, the AND / OR of the entries it writes to out (those below the
// prefix, and with take_all the equal ones it keeps) is merged into
// ctl->fin for the larger-K finish, which then needs no pass of its own.
template <bool FOLD>
__device__ void split_pass(const TopkArgs& a, bool cand, uint64_t src_n, uint64_t p0, uint64_t p1,
                           int L, int kb, bool take_all, uint64_t krem) {
    TopkCtl* ctl = a.ctl;
    uint64_t acc[4] = {~0ull, ~0ull, 0ull, 0ull};
    const uint64_t stride = static_cast<uint64_t>(TK_TPB) * gridDim.x;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t eq_base = a.k - krem;
    for (uint64_t wb = static_cast<uint64_t>(blockIdx.x) * TK_TPB + (threadIdx.x & ~31u); wb < src_n;
         wb += stride) {
        const uint64_t i = wb + lane;
        int c = 1;
        Elem e{0, 0};
        uint64_t w0 = 0, w1 = 0;
        if (i < src_n) {
            e = load_src(a, cand, i);
            comp_words(e.r, e.rid, kb, w0, w1);
            c = prefix_cmp(w0, w1, p0, p1, L);
        }
        const unsigned lt = __ballot_sync(0xFFFFFFFFu, c < 0);
        const unsigned eq = __ballot_sync(0xFFFFFFFFu, c == 0);
        if (lt) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctl->out_count, static_cast<unsigned long long>(__popc(lt)));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (c < 0) {
                const uint64_t pos = base + __popc(lt & ((1u << lane) - 1u));
                a.out_r0[pos] = e.r;
                a.out_rid0[pos] = e.rid;
                if (FOLD) and_or(w0, w1, acc);
            }
        }
        if (eq) {
            unsigned long long base = 0;
            unsigned long long* ctr = take_all ? &ctl->eq_count : &ctl->small_count;
            if (lane == 0) base = atomicAdd(ctr, static_cast<unsigned long long>(__popc(eq)));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (c == 0) {
                const uint64_t pos = base + __popc(eq & ((1u << lane) - 1u));
                if (take_all) {
                    if (pos < krem) {
                        a.out_r0[eq_base + pos] = e.r;
                        a.out_rid0[eq_base + pos] = e.rid;
                        if (FOLD) and_or(w0, w1, acc);
                    }
                } else if (pos < TK_SMALL) {
                    a.small_r[pos] = e.r;
                    a.small_rid[pos] = e.rid;
                }
            }
        }
    }
    if (FOLD) and_or_merge<TK_TPB>(acc, ctl->fin);
}

// Merge-path split: how many of the first `diag` outputs of the merge of
// A[0, na) and B[0, nb) come from A (A wins ties, keeping the merge stable).
__device__ __forceinline__ uint64_t merge_path(const uint64_t* ar, const uint32_t* arid, uint64_t na,
                                               const uint64_t* br, const uint32_t* brid, uint64_t nb,
                                               uint64_t diag) {
    uint64_t lo = diag > nb ? diag - nb : 0;
    uint64_t hi = diag < na ? diag : na;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        const uint64_t j = diag - 1 - mid;
        if (!elem_less(__ldcg(br + j), __ldcg(brid + j), __ldcg(ar + mid), __ldcg(arid + mid))) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Early exit after an expired wait: CTA 0 publishes the device status.
__device__ __forceinline__ void report(const TopkArgs& a) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.dev_status) *a.dev_status = ld_volatile_i32(&a.ctl->err);
}

}  // namespace

// Kernel 1 of 3: reset the control block and the histograms (CTA 0, and all
// CTAs' shares), and on the sampled path load the sample and estimate the
// filter threshold (TK_PREP_CTAS CTAs; the last one to finish selects).
__global__ void __launch_bounds__(TK_TPB) topk_prepare_kernel(TopkArgs a) {
    __shared__ unsigned sh[TK_BINS];
    __shared__ unsigned long long sc[24];
    __shared__ int last;
    TopkCtl* ctl = a.ctl;
    allow_next_grid();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->ts[0] = gtimer();
        ctl->cand_count = 0;
        ctl->out_count = 0;
        ctl->eq_count = 0;
        ctl->small_count = 0;
        ctl->err = 0;
        ctl->path = a.use_sample ? 1 : 0;
        ctl->passes = 0;
        ctl->thresh = ~0ull;
        for (int s = 0; s < 3; ++s) {
            ctl->ao[s][0] = ctl->ao[s][1] = ~0ull;
            ctl->ao[s][2] = ctl->ao[s][3] = 0ull;
        }
        ctl->fin[0] = ctl->fin[1] = ~0ull;
        ctl->fin[2] = ctl->fin[3] = 0ull;
    }
    for (int b = blockIdx.x * TK_TPB + threadIdx.x; b < 3 * TK_BINS; b += gridDim.x * TK_TPB) a.ghist[b] = 0;
    if (!a.use_sample) {
        if (threadIdx.x == 0) ctl->ts[1] = gtimer();
        return;
    }
    const uint64_t j = static_cast<uint64_t>(blockIdx.x) * TK_TPB + threadIdx.x;   // < TK_SAMPLE
    a.samples[j] = load_input(a, (j * a.n) / TK_SAMPLE + (a.n / TK_SAMPLE) / 2).r;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&a.bar->prep, 1u) + 1u) % gridDim.x == 0;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const uint64_t t = sample_threshold(a, sh, sc);
    if (threadIdx.x == 0) {
        ctl->thresh = t;
        ctl->ts[1] = gtimer();
    }
}

// Kernel 2 of 3 (sampled path only): the single streaming pass over the keys,
// bulk-copy flavour.  Independent CTAs, several per SM.
template <bool W4>
__global__ void __launch_bounds__(TKF_TPB, 4) topk_filter_bulk_kernel(TopkArgs a) {
    extern __shared__ __align__(128) unsigned char fsmem[];
    wait_prior_grid();
    const uint64_t t = __ldcg(&a.ctl->thresh);
    filter_pass_bulk<W4, TKF_TPB>(a, t, fsmem);
}

// Kernel 2 of 3, register-load flavour (TPB threads; the per-warp stages are
// dynamic shared memory, (TPB / 32) * WS_BYTES).
template <bool W4, int TPB>
__global__ void __launch_bounds__(TPB, 1024 / TPB) topk_filter_regs_kernel(TopkArgs a) {
    extern __shared__ __align__(16) unsigned char stage[];
    fuse_init<TPB>();
    wait_prior_grid();
    const uint64_t t = __ldcg(&a.ctl->thresh);
    filter_pass<W4, TPB>(a, t, stage);
    fuse_merge<TPB>(a);
}

// Kernel 2 of 3 for a two-column key (register loads of both columns).
template <int TPB>
__global__ void __launch_bounds__(TPB, 1024 / TPB) topk_filter_pair_kernel(TopkArgs a) {
    extern __shared__ __align__(16) unsigned char stage[];
    fuse_init<TPB>();
    wait_prior_grid();
    const uint64_t t = __ldcg(&a.ctl->thresh);
    filter_pass_pair<TPB>(a, t, stage);
    fuse_merge<TPB>(a);
}

// Kernel 3 of 3 (cooperative): refine, split, finish and sort.
__global__ void __launch_bounds__(TK_TPB, 2) topk_select_kernel(TopkArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long sc[24];
    TopkCtl* ctl = a.ctl;
    const int kb = a.w4 ? 32 : 64;
    const int TB = kb + 32;
    unsigned* sh = reinterpret_cast<unsigned*>(smem);
    uint64_t* sr = reinterpret_cast<uint64_t*>(smem);
    uint32_t* srid = reinterpret_cast<uint32_t*>(smem + TK_RANK_MAX * 8);

    wait_prior_grid();
    const bool stamp = blockIdx.x == 0 && threadIdx.x == 0;
    if (stamp) ctl->ts[2] = gtimer();
    // Source of the selection: the candidates of the streaming pass when the
    // sample judged well (at least k of them, all stored), else the input.
    bool cand = false;
    uint64_t src_n = a.n;
    if (a.use_sample) {
        if (ld_volatile_i32(&ctl->err) != 0) return report(a);
        const uint64_t cnt = __ldcg(&ctl->cand_count);
        cand = cnt >= a.k && cnt <= a.cand_cap;
        if (cand) src_n = cnt;
        if (stamp) ctl->path = cand ? 1 : 2;
    }
    const unsigned long long use_ts3 = stamp ? gtimer() : 0ull;

    // Phase 2: radix refine of the (rank word, row-id) prefix.  Candidates are
    // all at or below the threshold, so they share its leading zero bits: the
    // refine starts below them.
    uint64_t p0 = 0, p1 = 0, krem = a.k, bcnt = src_n;
    int L = 0, pass = 0, npass = 0;
    if (cand) {
        const int lz = __clzll(static_cast<long long>(__ldcg(&ctl->thresh)));
        L = lz < kb ? lz : kb;
    }
    // With the filter's fused first pass, pass 0's histogram is ready on the
    // candidate path; on the fallback path it holds the filter's partial
    // counts, so the passes start at buffer 1 (clean) and pass 2 clears
    // buffer 0 before pass 3 uses it.
    bool ready = a.fuse && cand;
    if (a.fuse && !cand) pass = 1;
    while (bcnt > TK_SMALL && L < TB && krem < bcnt) {
        const int d = min(a.digit, TB - L);
        unsigned* gh = a.ghist + (pass % 3) * TK_BINS;
        unsigned* gz = a.ghist + ((pass + 1) % 3) * TK_BINS;
        unsigned long long* ao = ctl->ao[pass % 3];
        const bool fused_pass = ready;
        if (!ready) {
            hist_pass(a, cand, src_n, p0, p1, L, d, kb, gh, gz, sh, ao, ctl->ao[(pass + 1) % 3]);
            if (!grid_sync(a.bar, &ctl->err)) return report(a);
        }
        ready = false;
        ++npass;
        const Pick pk = pick_bucket<TK_TPB>(gh, krem, sc);
        // every matching entry in one bucket (the fused pass folds no AND / OR)
        const bool whole = pk.below == 0 && pk.in_b == bcnt && !fused_pass;
        krem -= pk.below;
        bcnt = pk.in_b;
        prefix_set(p0, p1, L, d, pk.b);
        L += d;
        if (whole) {
            // The bucket holds exactly the entries the AND / OR saw: their
            // common bits join the prefix and the next digit starts where
            // they first differ.
            const int f = first_diff(ao, TB);
            if (f > L) {
                prefix_copy(p0, p1, __ldcg(ao + 0), __ldcg(ao + 1), L, f);
                L = f;
            }
        }
        ++pass;
    }
    // The buffer at pass % 3 must be clean for the finish: when the fused
    // pass-0 histogram was never consumed, buffer 1 (zeroed by prepare) is.
    if (ready) pass = 1;
    if (stamp) {
        ctl->passes = npass;
        ctl->ts[3] = use_ts3;
        ctl->ts[4] = gtimer();
    }

    // Phase 3: split around the prefix.
    const bool take_all = (krem == bcnt) || (L >= TB);
    // the larger-K finish wants the AND / OR of the entries split writes out
    const bool large = (take_all ? a.k : a.k - krem) + (take_all ? 0 : bcnt) > TK_RANK_MAX;
    if (large)
        split_pass<true>(a, cand, src_n, p0, p1, L, kb, take_all, krem);
    else
        split_pass<false>(a, cand, src_n, p0, p1, L, kb, take_all, krem);
    if (!grid_sync(a.bar, &ctl->err)) return report(a);
    if (stamp) ctl->ts[5] = gtimer();

    // Phase 4, survivors that fit one CTA's shared memory (every K <= 4096):
    // each warp of the grid takes survivors one at a time and computes its
    // final position as its rank -- the number of entries of its own set
    // that order before it (equal entries by position), so ranks are
    // distinct.  The "below" entries (prefix < P) precede every bucket entry;
    // a bucket entry is kept when its rank within the bucket is below krem.
    {
        const uint64_t nb = take_all ? a.k : a.k - krem;     // out_r0[0, nb)
        const uint64_t ns = take_all ? 0 : bcnt;             // small buffer
        if (nb + ns <= TK_RANK_MAX) {
            const int nbi = static_cast<int>(nb), nsi = static_cast<int>(ns);
            for (int i = threadIdx.x; i < nbi; i += TK_TPB) {
                sr[i] = __ldcg(a.out_r0 + i);
                srid[i] = __ldcg(a.out_rid0 + i);
            }
            for (int i = threadIdx.x; i < nsi; i += TK_TPB) {
                sr[nbi + i] = __ldcg(a.small_r + i);
                srid[nbi + i] = __ldcg(a.small_rid + i);
            }
            __syncthreads();
            if (stamp) ctl->ts[7] = gtimer();
            const unsigned lane = threadIdx.x & 31u;
            const int nwarps = static_cast<int>(gridDim.x) * (TK_TPB / 32);
            const int gw = static_cast<int>(blockIdx.x) * (TK_TPB / 32) + static_cast<int>(threadIdx.x >> 5);
            for (int e = gw; e < nbi + nsi; e += nwarps) {
                const bool below = e < nbi;
                const int lo = below ? 0 : nbi, hi = below ? nbi : nbi + nsi;
                const uint64_t er = sr[e];
                const uint32_t erid = srid[e];
                unsigned c = 0;
                for (int j = lo + static_cast<int>(lane); j < hi; j += 32) {
                    const uint64_t jr = sr[j];
                    const uint32_t jrid = srid[j];
                    c += (jr < er || (jr == er && (jrid < erid || (jrid == erid && j < e)))) ? 1u : 0u;
                }
                c = __reduce_add_sync(0xFFFFFFFFu, c);
                if (lane == 0) {
                    if (below) write_result(a, c, er, erid);
                    else if (c < krem) write_result(a, nb + c, er, erid);
                }
            }
            if (stamp) {
                ctl->ts[8] = gtimer();
                ctl->ts[6] = ctl->ts[8];
                if (a.dev_status) *a.dev_status = ld_volatile_i32(&ctl->err);
            }
            return;
        }
    }

    // Phase 4, larger K.  (a) The bucket entries (ns <= 4096) are ranked by
    // the grid as above and the first krem written at their final positions.
    // (b) The below entries are partitioned on the 12-bit digit at the refine
    // start L0 -- a histogram, a scan, a scatter into out_r1 -- and every
    // bucket of at most TK_SMALL entries is ranked in one CTA's shared memory
    // and written at its final positions.  Skewed inputs with a larger bucket
    // fall back to tile sorts and merge-path rounds.
    {
        const uint64_t nb = take_all ? a.k : a.k - krem;
        const int nsi = take_all ? 0 : static_cast<int>(bcnt);
        const unsigned lane = threadIdx.x & 31u;
        const int nwarps = static_cast<int>(gridDim.x) * (TK_TPB / 32);
        const int gw = static_cast<int>(blockIdx.x) * (TK_TPB / 32) + static_cast<int>(threadIdx.x >> 5);
        if (nsi > 0) {
            for (int i = threadIdx.x; i < nsi; i += TK_TPB) {
                sr[i] = __ldcg(a.small_r + i);
                srid[i] = __ldcg(a.small_rid + i);
            }
            __syncthreads();
            for (int e = gw; e < nsi; e += nwarps) {
                const uint64_t er = sr[e];
                const uint32_t erid = srid[e];
                unsigned c = 0;
                for (int j = static_cast<int>(lane); j < nsi; j += 32) {
                    const uint64_t jr = sr[j];
                    const uint32_t jrid = srid[j];
                    c += (jr < er || (jr == er && (jrid < erid || (jrid == erid && j < e)))) ? 1u : 0u;
                }
                c = __reduce_add_sync(0xFFFFFFFFu, c);
                if (lane == 0 && c < krem) write_result(a, nb + c, er, erid);
            }
            __syncthreads();
        }
        // (b) partition histogram of the below entries, on the digit that
        // starts at the first bit where they differ (their AND / OR, folded
        // by the split pass that wrote them), so that clustered keys and ties
        // on the key spread over the buckets.
        const int L0 = min(first_diff(ctl->fin, TB), TB - 1);
        const int dp = min(a.digit, TB - L0);
        unsigned* ph = a.ghist + (pass % 3) * TK_BINS;          // clean (zeroed by the last pass or prepare)
        unsigned* pc = a.ghist + ((pass + 1) % 3) * TK_BINS;    // cursors, zeroed here
        for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB) sh[b] = 0;
        if (blockIdx.x == 0)
            for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB) pc[b] = 0;
        __syncthreads();
        const uint64_t gstride = static_cast<uint64_t>(TK_TPB) * gridDim.x;
        for (uint64_t wb = static_cast<uint64_t>(blockIdx.x) * TK_TPB + (threadIdx.x & ~31u); wb < nb; wb += gstride) {
            const uint64_t i = wb + lane;
            unsigned dig = 0xFFFFFFFFu;
            if (i < nb) {
                uint64_t w0, w1;
                comp_words(__ldcg(a.out_r0 + i), __ldcg(a.out_rid0 + i), kb, w0, w1);
                dig = comp_digit(w0, w1, L0, dp);
            }
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
            if (dig != 0xFFFFFFFFu && lane == static_cast<unsigned>(__ffs(peers) - 1))
                atomicAdd(&sh[dig], static_cast<unsigned>(__popc(peers)));
        }
        __syncthreads();
        for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB)
            if (sh[b]) atomicAdd(&ph[b], sh[b]);
        if (!grid_sync(a.bar, &ctl->err)) return report(a);
        // Scan of the partition histogram (every CTA), largest bucket.
        constexpr int PER = TK_BINS / TK_TPB;
        unsigned v[PER];
        unsigned long long local = 0;
        unsigned mx = 0;
        const volatile unsigned* hv = ph;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            v[j] = hv[threadIdx.x * PER + j];
            local += v[j];
            mx = max(mx, v[j]);
        }
        const unsigned long long before = block_excl_scan<TK_TPB>(local, reinterpret_cast<unsigned long long*>(sc),
                                                          reinterpret_cast<unsigned long long*>(sc) + 16);
        unsigned* off = sh;                                      // exclusive offsets per bucket
        {
            unsigned long long run = before;
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                off[threadIdx.x * PER + j] = static_cast<unsigned>(run);
                run += v[j];
            }
        }
        const bool fits = __syncthreads_and(mx <= static_cast<unsigned>(TK_SMALL));
        if (fits) {
            // Scatter the below entries into bucket order (out_r1).
            for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * TK_TPB + threadIdx.x; i < nb; i += gstride) {
                const uint64_t er = __ldcg(a.out_r0 + i);
                const uint32_t erid = __ldcg(a.out_rid0 + i);
                uint64_t w0, w1;
                comp_words(er, erid, kb, w0, w1);
                const unsigned d = comp_digit(w0, w1, L0, dp);
                const unsigned pos = off[d] + atomicAdd(&pc[d], 1u);
                a.out_r1[pos] = er;
                a.out_rid1[pos] = erid;
            }
            if (!grid_sync(a.bar, &ctl->err)) return report(a);
            // Buckets of at most 32 entries: one warp each, ranked in
            // registers (lane i holds entry i; the others come by shuffle).
            for (int b = gw; b < TK_BINS; b += nwarps) {
                const unsigned m = hv[b];
                if (m == 0 || m > 32) continue;
                const unsigned o = off[b];
                uint64_t er = 0;
                uint32_t erid = 0;
                if (lane < m) {
                    er = __ldcg(a.out_r1 + o + lane);
                    erid = __ldcg(a.out_rid1 + o + lane);
                }
                unsigned c = 0;
                for (unsigned j = 0; j < m; ++j) {
                    const uint64_t jr = __shfl_sync(0xFFFFFFFFu, er, j);
                    const uint32_t jrid = __shfl_sync(0xFFFFFFFFu, erid, j);
                    c += (jr < er || (jr == er && (jrid < erid || (jrid == erid && j < lane)))) ? 1u : 0u;
                }
                if (lane < m) write_result(a, o + c, er, erid);
            }
            // Larger buckets: one CTA each, ranked in shared memory.
            uint64_t* br = reinterpret_cast<uint64_t*>(smem + TK_BINS * 4);
            uint32_t* brid = reinterpret_cast<uint32_t*>(smem + TK_BINS * 4 + TK_SMALL * 8);
            for (int b = blockIdx.x; b < TK_BINS; b += gridDim.x) {
                const unsigned m = hv[b];
                if (m <= 32) continue;
                const unsigned o = off[b];
                for (unsigned i = threadIdx.x; i < m; i += TK_TPB) {
                    br[i] = __ldcg(a.out_r1 + o + i);
                    brid[i] = __ldcg(a.out_rid1 + o + i);
                }
                __syncthreads();
                for (unsigned e = threadIdx.x >> 5; e < m; e += TK_TPB / 32) {
                    const uint64_t er = br[e];
                    const uint32_t erid = brid[e];
                    unsigned c = 0;
                    for (unsigned j = lane; j < m; j += 32) {
                        const uint64_t jr = br[j];
                        const uint32_t jrid = brid[j];
                        c += (jr < er || (jr == er && (jrid < erid || (jrid == erid && j < e)))) ? 1u : 0u;
                    }
                    c = __reduce_add_sync(0xFFFFFFFFu, c);
                    if (lane == 0) write_result(a, o + c, er, erid);
                }
                __syncthreads();
            }
            if (stamp) {
                ctl->ts[7] = gtimer();
                ctl->ts[8] = ctl->ts[7];
                ctl->ts[6] = ctl->ts[7];
                if (a.dev_status) *a.dev_status = ld_volatile_i32(&ctl->err);
            }
            return;
        }
        // Skewed: the bucket entries are already written; sort the below
        // entries with the merge path (k below plus krem written above).
    }

    // Phase 4, fallback: CTA 0 finishes the bucket, then a grid merge sort.
    if (blockIdx.x == 0) {
        if (!take_all) {
            const int cnt = static_cast<int>(bcnt);
            for (int i = threadIdx.x; i < cnt; i += TK_TPB) {
                sr[i] = __ldcg(a.small_r + i);
                srid[i] = __ldcg(a.small_rid + i);
            }
            __syncthreads();
            block_sort<TK_TPB>(sr, srid, cnt);
            const uint64_t base = a.k - krem;
            for (uint64_t i = threadIdx.x; i < krem; i += TK_TPB) {
                a.out_r0[base + i] = sr[i];
                a.out_rid0[base + i] = srid[i];
            }
            __syncthreads();
        }
        if (stamp) ctl->ts[7] = gtimer();
        if (a.k <= TK_SMALL) {
            const int cnt = static_cast<int>(a.k);
            for (int i = threadIdx.x; i < cnt; i += TK_TPB) {
                sr[i] = __ldcg(a.out_r0 + i);
                srid[i] = __ldcg(a.out_rid0 + i);
            }
            __syncthreads();
            block_sort<TK_TPB>(sr, srid, cnt);
            if (stamp) ctl->ts[8] = gtimer();
            for (int i = threadIdx.x; i < cnt; i += TK_TPB) write_result(a, i, sr[i], srid[i]);
            if (threadIdx.x == 0 && a.dev_status) *a.dev_status = ld_volatile_i32(&ctl->err);
            if (threadIdx.x == 0) ctl->ts[6] = gtimer();
        }
    }
    if (a.k <= TK_SMALL) return;
    if (!grid_sync(a.bar, &ctl->err)) return report(a);

    // K > 4096: sort tiles of TK_SMALL, then merge-path rounds.
    const uint64_t k = a.k;
    const uint64_t ntiles = (k + TK_SMALL - 1) / TK_SMALL;
    for (uint64_t tIdx = blockIdx.x; tIdx < ntiles; tIdx += gridDim.x) {
        const uint64_t lo = tIdx * TK_SMALL;
        const int cnt = static_cast<int>(k - lo < TK_SMALL ? k - lo : TK_SMALL);
        for (int i = threadIdx.x; i < cnt; i += TK_TPB) {
            sr[i] = __ldcg(a.out_r0 + lo + i);
            srid[i] = __ldcg(a.out_rid0 + lo + i);
        }
        __syncthreads();
        block_sort<TK_TPB>(sr, srid, cnt);
        for (int i = threadIdx.x; i < cnt; i += TK_TPB) {
            a.out_r0[lo + i] = sr[i];
            a.out_rid0[lo + i] = srid[i];
        }
        __syncthreads();
    }
    if (!grid_sync(a.bar, &ctl->err)) return report(a);
    uint64_t* src_r = a.out_r0;
    uint32_t* src_rid = a.out_rid0;
    uint64_t* dst_r = a.out_r1;
    uint32_t* dst_rid = a.out_rid1;
    constexpr uint64_t E = 8;
    const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * TK_TPB;
    const uint64_t gtid = static_cast<uint64_t>(blockIdx.x) * TK_TPB + threadIdx.x;
    for (uint64_t w = TK_SMALL; w < k; w *= 2) {
        const uint64_t ntasks = (k + E - 1) / E;
        for (uint64_t task = gtid; task < ntasks; task += nthreads) {
            const uint64_t o = task * E;
            const uint64_t base = (o / (2 * w)) * (2 * w);
            const uint64_t a0 = base, a1 = min(base + w, k);
            const uint64_t b0 = a1, b1 = min(base + 2 * w, k);
            const uint64_t na = a1 - a0, nb = b1 - b0;
            const uint64_t diag = o - base;
            uint64_t i = merge_path(src_r + a0, src_rid + a0, na, src_r + b0, src_rid + b0, nb, diag);
            uint64_t j = diag - i;
            const uint64_t end = min(o + E, b1);
            uint64_t ar = 0, br = 0;
            uint32_t arid = 0, brid = 0;
            if (i < na) { ar = __ldcg(src_r + a0 + i); arid = __ldcg(src_rid + a0 + i); }
            if (j < nb) { br = __ldcg(src_r + b0 + j); brid = __ldcg(src_rid + b0 + j); }
            for (uint64_t q = o; q < end; ++q) {
                const bool takeA = i < na && (j >= nb || !elem_less(br, brid, ar, arid));
                if (takeA) {
                    dst_r[q] = ar;
                    dst_rid[q] = arid;
                    ++i;
                    if (i < na) { ar = __ldcg(src_r + a0 + i); arid = __ldcg(src_rid + a0 + i); }
                } else {
                    dst_r[q] = br;
                    dst_rid[q] = brid;
                    ++j;
                    if (j < nb) { br = __ldcg(src_r + b0 + j); brid = __ldcg(src_rid + b0 + j); }
                }
            }
        }
        if (!grid_sync(a.bar, &ctl->err)) return report(a);
        uint64_t* tr = src_r; src_r = dst_r; dst_r = tr;
        uint32_t* ti = src_rid; src_rid = dst_rid; dst_rid = ti;
    }
    for (uint64_t i = gtid; i < k; i += nthreads) write_result(a, i, __ldcg(src_r + i), __ldcg(src_rid + i));
    if (gtid == 0 && a.dev_status) *a.dev_status = ld_volatile_i32(&ctl->err);
    if (gtid == 0) ctl->ts[6] = gtimer();
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
TopkPlan topk_plan(uint64_t n, uint64_t k) {
    TopkPlan p{0, 0, 0};
    if (n > TK_DIRECT_N && k <= n / 256) {
        const double lam = static_cast<double>(k) * TK_SAMPLE / static_cast<double>(n);
        double r = std::ceil(lam + 4.0 * std::sqrt(lam)) + 3.0;
        if (r > TK_SAMPLE) r = TK_SAMPLE;
        p.use_sample = 1;
        p.sample_rank = static_cast<unsigned>(r);
        const uint64_t stratum = (n + TK_SAMPLE - 1) / TK_SAMPLE;
        uint64_t cap = 2 * (static_cast<uint64_t>(r) + 8) * stratum;
        cap = std::max<uint64_t>(cap, k + TK_SMALL);
        cap = (cap + 1023) & ~1023ull;
        p.cand_cap = std::min<uint64_t>(cap, n);
    }
    return p;
}

static size_t up256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

size_t topk_scratch_bytes(const TopkPlan& p, uint64_t k) {
    size_t b = up256(sizeof(TopkCtl)) + up256(sizeof(GridBar)) + up256(3 * TK_BINS * 4);
    if (p.use_sample) b += up256(TK_SAMPLE * 8);
    b += up256(p.cand_cap * 8) + up256(p.cand_cap * 4);
    b += up256(TK_SMALL * 8) + up256(TK_SMALL * 4);
    const uint64_t kk = std::max<uint64_t>(k, 1);
    b += up256(kk * 8) + up256(kk * 4);
    if (k > TK_SMALL) b += up256(kk * 8) + up256(kk * 4);
    return b;
}

void topk_carve(TopkArgs& a, const TopkPlan& p, void* base) {
    unsigned char* c = static_cast<unsigned char*>(base);
    auto take = [&](size_t bytes) {
        void* r = c;
        c += up256(bytes);
        return r;
    };
    // The grid barrier comes first so that it keeps its place (and its
    // zeroed state) whatever the other buffer sizes are.
    a.bar = static_cast<GridBar*>(take(sizeof(GridBar)));
    a.ctl = static_cast<TopkCtl*>(take(sizeof(TopkCtl)));
    a.ghist = static_cast<unsigned*>(take(3 * TK_BINS * 4));
    a.small_r = static_cast<uint64_t*>(take(TK_SMALL * 8));
    a.small_rid = static_cast<uint32_t*>(take(TK_SMALL * 4));
    a.cand_cap = p.cand_cap;
    a.cand_r = static_cast<uint64_t*>(take(p.cand_cap * 8));
    a.cand_rid = static_cast<uint32_t*>(take(p.cand_cap * 4));
    const uint64_t kk = std::max<uint64_t>(a.k, 1);
    a.out_r0 = static_cast<uint64_t*>(take(kk * 8));
    a.out_rid0 = static_cast<uint32_t*>(take(kk * 4));
    if (a.k > TK_SMALL) {
        a.out_r1 = static_cast<uint64_t*>(take(kk * 8));
        a.out_rid1 = static_cast<uint32_t*>(take(kk * 4));
    } else {
        a.out_r1 = nullptr;
        a.out_rid1 = nullptr;
    }
    a.samples = p.use_sample ? static_cast<uint64_t*>(take(TK_SAMPLE * 8)) : nullptr;
    a.use_sample = p.use_sample;
    a.sample_rank = p.sample_rank;
    a.filter = TK_FILTER_BULK;
}

// Dynamic shared bytes the filter kernel may use, per device; set once, under
// g_attr_lock, by the first thread that needs the kernels' attributes there.
static std::atomic<int> g_smem_limit[64] = {};
static std::mutex g_attr_lock;

static bool set_kernel_attrs(int device) {
    if (g_smem_limit[device].load()) return true;
    std::lock_guard<std::mutex> guard(g_attr_lock);
    if (g_smem_limit[device].load()) return true;
    // Opt-in limit per block, less the filter kernel's static shared memory.
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, topk_filter_bulk_kernel<false>) != cudaSuccess)
        return false;
    const int lim = std::min<int>(optin - static_cast<int>(fa.sharedSizeBytes) - 256, TK_SMEM_MAX);
    if (cudaFuncSetAttribute(topk_filter_bulk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             lim) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_bulk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             lim) != cudaSuccess ||
        // the register filters' stages are dynamic, next to the fused pass's
        // static histogram: above 48 KB together, so every variant opts in
        cudaFuncSetAttribute(topk_filter_regs_kernel<false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             8 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_regs_kernel<true, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             8 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_pair_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             8 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_regs_kernel<false, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             16 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_regs_kernel<true, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             16 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_pair_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             16 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_regs_kernel<false, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             32 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_regs_kernel<true, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             32 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_filter_pair_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             32 * WS_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(topk_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TK_SORT_SMEM) != cudaSuccess)
        return false;
    g_smem_limit[device].store(lim);
    return true;
}

bool topk_geometry(int device, int tile_bytes, int stages, int ctas_per_sm, int regs_tpb, TopkGeom* out) {
    TopkGeom g;
    g.regs_tpb = regs_tpb ? regs_tpb : TKR_TPB;
    if (g.regs_tpb != 256 && g.regs_tpb != 512 && g.regs_tpb != 1024) return false;
    g.tile_bytes = tile_bytes ? tile_bytes : TK_TILE_DEFAULT;
    g.stages = stages ? stages : TK_STAGES_DEFAULT;
    g.ctas_per_sm = ctas_per_sm ? ctas_per_sm : TK_CTAS_PER_SM_DEFAULT;
    if (g.tile_bytes < 16 * TKF_TPB || g.tile_bytes % (16 * TKF_TPB) || g.stages < 1 ||
        g.stages > TK_MAX_STAGES || g.ctas_per_sm < 1 || g.ctas_per_sm > 8)
        return false;
    if (device < 0 || device >= 64) return false;
    g.smem_bytes = g.tile_bytes * g.stages + 16 * TK_MAX_STAGES + (TKF_TPB / 32) * WS_BYTES;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return false;
    if (!set_kernel_attrs(device)) return false;
    if (g.smem_bytes > g_smem_limit[device].load()) return false;
    // Streaming filter: independent CTAs, capped at ctas_per_sm per SM.
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_filter_bulk_kernel<false>, TKF_TPB,
                                                      g.smem_bytes) != cudaSuccess)
        return false;
    per_sm = std::min(per_sm, g.ctas_per_sm);
    if (per_sm < 1) return false;
    g.filter_grid = sms * per_sm;
    cudaError_t oe;
    const size_t rs = static_cast<size_t>(g.regs_tpb / 32) * WS_BYTES;
    if (g.regs_tpb == 256)
        oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_filter_regs_kernel<false, 256>, 256, rs);
    else if (g.regs_tpb == 512)
        oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_filter_regs_kernel<false, 512>, 512, rs);
    else
        oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_filter_regs_kernel<false, 1024>, 1024, rs);
    if (oe != cudaSuccess) return false;
    g.regs_grid = sms * std::max(1, std::min(per_sm, 2048 / g.regs_tpb));
    // Cooperative select kernel: every CTA resident, two per SM at most.
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_select_kernel, TK_TPB, TK_SORT_SMEM) !=
        cudaSuccess)
        return false;
    // Two CTAs per SM for the select in general; one per SM when it reads a
    // candidate list and finishes a small K: its grid barriers then dominate,
    // and half the arrivals take less time (measured, 2^28 keys, K = 1000:
    // select 22.6 -> 19.9 us; at K = 10^5 the merge-path finish wants both).
    per_sm = std::min(per_sm, 2);
    if (per_sm < 1) return false;
    g.grid = sms * per_sm;
    g.grid_small = sms;
    *out = g;
    return true;
}

// One launch of a Top-K kernel: cooperative for the select, and with
// programmatic stream serialisation (the kernel waits in wait_prior_grid for
// the one before it).
static cudaError_t launch_kernel(void (*fn)(TopkArgs), unsigned grid, unsigned block, size_t smem,
                                 cudaStream_t stream, const TopkArgs& a, bool coop) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[2];
    unsigned na = 0;
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
    if (coop) {
        at[na].id = cudaLaunchAttributeCooperative;
        at[na].val.cooperative = 1;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

cudaError_t topk_launch(const TopkArgs& args, const TopkGeom& geom, cudaStream_t stream, cudaEvent_t* ev) {
    TopkArgs a = args;
    a.tile_bytes = geom.tile_bytes;
    a.stages = geom.stages;
    if (a.digit == 0) a.digit = TK_DIG;
    if (a.digit < TK_DIG_MIN || a.digit > TK_DIG) return cudaErrorInvalidValue;
    // the register and two-column filters fold the select's first pass
    a.fuse = a.use_sample && (a.pair || a.filter == TK_FILTER_REGS) ? 1 : 0;
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], stream)) != cudaSuccess) return e;
    topk_prepare_kernel<<<a.use_sample ? TK_PREP_CTAS : 1, TK_TPB, 0, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], stream)) != cudaSuccess) return e;
    if (a.use_sample) {
        void (*fn)(TopkArgs) = nullptr;
        unsigned grid = static_cast<unsigned>(geom.regs_grid), block = static_cast<unsigned>(geom.regs_tpb);
        size_t smem = static_cast<size_t>(geom.regs_tpb / 32) * WS_BYTES;
        if (a.pair) {
            fn = geom.regs_tpb == 256    ? topk_filter_pair_kernel<256>
                 : geom.regs_tpb == 1024 ? topk_filter_pair_kernel<1024>
                                         : topk_filter_pair_kernel<512>;
        } else if (a.filter == TK_FILTER_REGS) {
            if (geom.regs_tpb == 256)
                fn = a.w4 ? topk_filter_regs_kernel<true, 256> : topk_filter_regs_kernel<false, 256>;
            else if (geom.regs_tpb == 1024)
                fn = a.w4 ? topk_filter_regs_kernel<true, 1024> : topk_filter_regs_kernel<false, 1024>;
            else
                fn = a.w4 ? topk_filter_regs_kernel<true, 512> : topk_filter_regs_kernel<false, 512>;
        } else {
            fn = a.w4 ? topk_filter_bulk_kernel<true> : topk_filter_bulk_kernel<false>;
            grid = static_cast<unsigned>(geom.filter_grid);
            block = TKF_TPB;
            smem = geom.smem_bytes;
        }
        if ((e = launch_kernel(fn, grid, block, smem, stream, a, false)) != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[2], stream)) != cudaSuccess) return e;
    // (the direct path keeps both CTAs per SM: at 2^20 keys one per SM was
    // measured slower, 0.051 against 0.049 ms)
    const int sgrid = (a.use_sample && a.k <= static_cast<uint64_t>(TK_SMALL)) ? geom.grid_small : geom.grid;
    e = launch_kernel(topk_select_kernel, static_cast<unsigned>(sgrid), TK_TPB, TK_SORT_SMEM, stream, a, true);
    if (e != cudaSuccess || !ev) return e;
    return cudaEventRecord(ev[3], stream);
}

}  // namespace olap
