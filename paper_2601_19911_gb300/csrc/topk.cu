// Top-K selection over key-only (key, row-id) columns: ORDER BY key LIMIT K
// (Sec. III-A, "partial selection (or radix-based selection)", returning the
// row pointers of the Top-K rows in order).
//
// One cooperative launch runs the whole selection; CTAs meet at bounded grid
// barriers between phases:
//   0. (N > 2^21, K small against N) CTA 0 reads a stratified sample of 8192
//      keys and finds the rank word of the sample's r-th best entry by an
//      in-register radix select; r is chosen so that, with high probability,
//      at least K keys but not many more fall at or below it.
//   1. Filter: the only full pass over the keys.  16-byte streaming loads,
//      order-preserving transform in registers, and every rank word at or
//      below the threshold is appended (warp-aggregated) to a candidate
//      buffer with its row-id.  If the sample misjudged (fewer than K
//      candidates, or more than the buffer holds) the later phases run on
//      the full input instead.
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
#include <cmath>

#include "topk.cuh"

namespace olap {

namespace {

struct Elem {
    uint64_t r;
    uint32_t rid;
};

__device__ __forceinline__ bool elem_less(uint64_t ar, uint32_t arid, uint64_t br, uint32_t brid) {
    return ar < br || (ar == br && arid < brid);
}

__device__ __forceinline__ Elem load_input(const TopkArgs& a, uint64_t i) {
    Elem e;
    if (a.f32)
        e.r = rank_f32(static_cast<const uint32_t*>(a.keys)[i], a.desc);
    else
        e.r = rank_i64(static_cast<const uint64_t*>(a.keys)[i], a.desc);
    e.rid = a.rowids ? a.rowids[i] : static_cast<uint32_t>(i);
    return e;
}

__device__ __forceinline__ Elem load_src(const TopkArgs& a, bool cand, uint64_t i) {
    if (cand) return Elem{__ldcg(a.cand_r + i), __ldcg(a.cand_rid + i)};
    return load_input(a, i);
}

__device__ __forceinline__ uint4 ld_stream_v4(const void* p) {
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Block-wide exclusive scan helper over one value per thread (TK_TPB threads).
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
        constexpr int NW = TK_TPB / 32;
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

// Find the bucket b of a TK_BINS histogram where the running count first
// reaches `need` (1 <= need <= total).  Every thread gets b, the count below b
// and the count in b.
struct Pick {
    unsigned b;
    unsigned long long below;
    unsigned long long in_b;
};

__device__ Pick pick_bucket(const unsigned* hist, unsigned long long need, unsigned long long* sc) {
    constexpr int PER = TK_BINS / TK_TPB;   // 8 bins per thread
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
    const unsigned long long before = block_excl_scan(local, warp_sums, total);
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

// Bitonic sort of `count` (<= TK_SMALL) entries in shared memory, ascending
// by (r, rid); padded to a power of two with all-ones entries.
__device__ void block_sort(uint64_t* sr, uint32_t* srid, int count) {
    int m = 1;
    while (m < count) m <<= 1;
    for (int i = count + threadIdx.x; i < m; i += TK_TPB) {
        sr[i] = ~0ull;
        srid[i] = ~0u;
    }
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (m >> 1); t += TK_TPB) {
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

__device__ __forceinline__ void write_result(const TopkArgs& a, uint64_t i, uint64_t r, uint32_t rid) {
    if (a.f32)
        static_cast<uint32_t*>(a.out_keys)[i] = unrank_f32(r, a.desc);
    else
        static_cast<uint64_t*>(a.out_keys)[i] = unrank_i64(r, a.desc);
    a.out_rowids[i] = rid;
}

// Phase 0 (CTA 0): rank word of the sample's r-th smallest entry.
__device__ uint64_t sample_threshold(const TopkArgs& a, unsigned* sh, unsigned long long* sc) {
    uint64_t s[TK_SPT];
    const uint64_t n = a.n;
#pragma unroll
    for (int j = 0; j < TK_SPT; ++j) {
        const uint64_t idx = static_cast<uint64_t>(j) * TK_TPB + threadIdx.x;
        const uint64_t pos = (idx * n) / TK_SAMPLE + (n / TK_SAMPLE) / 2;
        s[j] = load_input(a, pos).r;
    }
    const int kb = a.f32 ? 32 : 64;
    uint64_t prefix = 0;
    unsigned long long rem = a.sample_rank;
    for (int L = 0; L < kb; L += 8) {
        for (int b = threadIdx.x; b < 256; b += TK_TPB) sh[b] = 0;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TK_SPT; ++j) {
            const bool match = (L == 0) || (((s[j] ^ prefix) >> (64 - L)) == 0);
            if (match) atomicAdd(&sh[(s[j] >> (56 - L)) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const unsigned lane = threadIdx.x;
            unsigned v[8];
            unsigned loc = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = sh[lane * 8 + j];
                loc += v[j];
            }
            unsigned incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= static_cast<unsigned>(o)) incl += t;
            }
            unsigned run = incl - loc;
            if (run < rem && rem <= run + loc) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (run < rem && rem <= run + v[j]) {
                        sc[0] = lane * 8 + j;
                        sc[1] = run;
                    }
                    run += v[j];
                }
            }
        }
        __syncthreads();
        prefix |= static_cast<uint64_t>(sc[0]) << (56 - L);
        rem -= sc[1];
        __syncthreads();
    }
    return prefix;
}

// Phase 1: the single streaming pass.  Appends (rank word, row-id) of every
// key whose rank word is <= t; counts all of them.
template <bool F32>
__device__ void filter_pass(const TopkArgs& a, uint64_t t) {
    constexpr int W = F32 ? 4 : 8;
    constexpr int VEC = 16 / W;
    TopkCtl* ctl = a.ctl;
    const uint64_t n = a.n;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(a.keys);
    const uint64_t head0 = ((16 - (addr & 15)) & 15) / W;
    const uint64_t head = head0 < n ? head0 : n;
    const uint64_t nvec = (n - head) / VEC;
    const uint64_t tail0 = head + nvec * VEC;
    const unsigned char* vbase = static_cast<const unsigned char*>(a.keys) + head * W;

    auto emit = [&](unsigned cnt, const uint64_t* rs, const uint64_t* idxs) {
        const unsigned long long pos = warp_append(&ctl->cand_count, cnt);
        for (unsigned j = 0; j < cnt; ++j) {
            if (pos + j < a.cand_cap) {
                a.cand_r[pos + j] = rs[j];
                a.cand_rid[pos + j] = a.rowids ? a.rowids[idxs[j]] : static_cast<uint32_t>(idxs[j]);
            }
        }
    };

    const uint64_t per_block = static_cast<uint64_t>(TK_TPB) * TK_UNROLL;
    const uint64_t stride = per_block * gridDim.x;
    for (uint64_t bb = per_block * blockIdx.x; bb < nvec; bb += stride) {
        uint4 v[TK_UNROLL];
#pragma unroll
        for (int u = 0; u < TK_UNROLL; ++u) {
            const uint64_t vi = bb + static_cast<uint64_t>(u) * TK_TPB + threadIdx.x;
            if (vi < nvec) v[u] = ld_stream_v4(vbase + vi * 16);
            else v[u] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        }
        uint64_t rs[TK_UNROLL * VEC];
        unsigned hit = 0;
#pragma unroll
        for (int u = 0; u < TK_UNROLL; ++u) {
            const uint64_t vi = bb + static_cast<uint64_t>(u) * TK_TPB + threadIdx.x;
            const bool ok = vi < nvec;
            if (F32) {
                const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    rs[u * 4 + e] = rank_f32(w[e], a.desc);
                    if (ok && rs[u * 4 + e] <= t) hit |= 1u << (u * 4 + e);
                }
            } else {
                const uint64_t w0 = static_cast<uint64_t>(v[u].x) | (static_cast<uint64_t>(v[u].y) << 32);
                const uint64_t w1 = static_cast<uint64_t>(v[u].z) | (static_cast<uint64_t>(v[u].w) << 32);
                rs[u * 2 + 0] = rank_i64(w0, a.desc);
                rs[u * 2 + 1] = rank_i64(w1, a.desc);
                if (ok && rs[u * 2 + 0] <= t) hit |= 1u << (u * 2 + 0);
                if (ok && rs[u * 2 + 1] <= t) hit |= 1u << (u * 2 + 1);
            }
        }
        if (__any_sync(0xFFFFFFFFu, hit != 0)) {
            uint64_t hr[TK_UNROLL * VEC], hi[TK_UNROLL * VEC];
            unsigned c = 0;
#pragma unroll
            for (int j = 0; j < TK_UNROLL * VEC; ++j) {
                if (hit & (1u << j)) {
                    const int u = j / VEC, e = j % VEC;
                    const uint64_t vi = bb + static_cast<uint64_t>(u) * TK_TPB + threadIdx.x;
                    hr[c] = rs[j];
                    hi[c] = head + vi * VEC + e;
                    ++c;
                }
            }
            emit(c, hr, hi);
        }
    }
    // Unaligned head and ragged tail: at most 2*VEC - 2 keys, one per lane of
    // warp 0 of CTA 0.
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const uint64_t rest = head + (n - tail0);
        const uint64_t j = threadIdx.x;
        uint64_t r = 0, idx = 0;
        unsigned c = 0;
        if (j < rest) {
            idx = j < head ? j : tail0 + (j - head);
            r = load_input(a, idx).r;
            c = r <= t ? 1u : 0u;
        }
        emit(c, &r, &idx);
    }
}

// One refine pass: histogram of digit [L, L+d) of the composites that match
// the prefix, merged into `gh`.  `gz` (another buffer) is cleared by CTA 0.
__device__ void hist_pass(const TopkArgs& a, bool cand, uint64_t src_n, uint64_t p0, uint64_t p1,
                          int L, int d, int kb, unsigned* gh, unsigned* gz, unsigned* sh) {
    for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB) sh[b] = 0;
    if (blockIdx.x == 0)
        for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB) gz[b] = 0;
    __syncthreads();
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
            if (prefix_cmp(w0, w1, p0, p1, L) == 0) dig = comp_digit(w0, w1, L, d);
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, dig);
        if (dig != 0xFFFFFFFFu && lane == static_cast<unsigned>(__ffs(peers) - 1))
            atomicAdd(&sh[dig], static_cast<unsigned>(__popc(peers)));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < TK_BINS; b += TK_TPB)
        if (sh[b]) atomicAdd(&gh[b], sh[b]);
}

// Split: entries below the prefix are selected (appended to out), entries
// equal to it go to the small buffer, or straight to out when all of them
// (or any `krem` identical ones) are taken.
__device__ void split_pass(const TopkArgs& a, bool cand, uint64_t src_n, uint64_t p0, uint64_t p1,
                           int L, int kb, bool take_all, uint64_t krem) {
    TopkCtl* ctl = a.ctl;
    const uint64_t stride = static_cast<uint64_t>(TK_TPB) * gridDim.x;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t eq_base = a.k - krem;
    for (uint64_t wb = static_cast<uint64_t>(blockIdx.x) * TK_TPB + (threadIdx.x & ~31u); wb < src_n;
         wb += stride) {
        const uint64_t i = wb + lane;
        int c = 1;
        Elem e{0, 0};
        if (i < src_n) {
            e = load_src(a, cand, i);
            uint64_t w0, w1;
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
                    }
                } else if (pos < TK_SMALL) {
                    a.small_r[pos] = e.r;
                    a.small_rid[pos] = e.rid;
                }
            }
        }
    }
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

__global__ void __launch_bounds__(TK_TPB, 2) topk_kernel(TopkArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long sc[24];
    TopkCtl* ctl = a.ctl;
    const int kb = a.f32 ? 32 : 64;
    const int TB = kb + 32;
    unsigned* sh = reinterpret_cast<unsigned*>(smem);
    uint64_t* sr = reinterpret_cast<uint64_t*>(smem);
    uint32_t* srid = reinterpret_cast<uint32_t*>(smem + TK_SMALL * 8);

    // Phase 0: reset the control block and histograms; estimate the threshold.
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            ctl->cand_count = 0;
            ctl->out_count = 0;
            ctl->eq_count = 0;
            ctl->small_count = 0;
            ctl->err = 0;
            ctl->path = a.use_sample ? 1 : 0;
            ctl->passes = 0;
        }
        for (int b = threadIdx.x; b < 3 * TK_BINS; b += TK_TPB) a.ghist[b] = 0;
        if (a.use_sample) {
            const uint64_t t = sample_threshold(a, sh, sc);
            if (threadIdx.x == 0) ctl->thresh = t;
        }
    }
    if (!grid_sync(a.bar, &ctl->err)) return report(a);

    // Phase 1: one streaming pass that keeps the keys at or below the threshold.
    bool cand = false;
    uint64_t src_n = a.n;
    if (a.use_sample) {
        const uint64_t t = *reinterpret_cast<volatile unsigned long long*>(&ctl->thresh);
        if (a.f32) filter_pass<true>(a, t);
        else filter_pass<false>(a, t);
        if (!grid_sync(a.bar, &ctl->err)) return report(a);
        const uint64_t cnt = *reinterpret_cast<volatile unsigned long long*>(&ctl->cand_count);
        cand = cnt >= a.k && cnt <= a.cand_cap;
        if (cand) src_n = cnt;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->path = cand ? 1 : 2;
    }

    // Phase 2: radix refine of the (rank word, row-id) prefix.
    uint64_t p0 = 0, p1 = 0, krem = a.k, bcnt = src_n;
    int L = 0, pass = 0;
    while (bcnt > TK_SMALL && L < TB && krem < bcnt) {
        const int d = min(TK_DIG, TB - L);
        unsigned* gh = a.ghist + (pass % 3) * TK_BINS;
        unsigned* gz = a.ghist + ((pass + 1) % 3) * TK_BINS;
        hist_pass(a, cand, src_n, p0, p1, L, d, kb, gh, gz, sh);
        if (!grid_sync(a.bar, &ctl->err)) return report(a);
        const Pick pk = pick_bucket(gh, krem, sc);
        krem -= pk.below;
        bcnt = pk.in_b;
        prefix_set(p0, p1, L, d, pk.b);
        L += d;
        ++pass;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->passes = pass;

    // Phase 3: split around the prefix.
    const bool take_all = (krem == bcnt) || (L >= TB);
    split_pass(a, cand, src_n, p0, p1, L, kb, take_all, krem);
    if (!grid_sync(a.bar, &ctl->err)) return report(a);

    // Phase 4: finish and sort.
    if (blockIdx.x == 0) {
        if (!take_all) {
            const int cnt = static_cast<int>(bcnt);
            for (int i = threadIdx.x; i < cnt; i += TK_TPB) {
                sr[i] = __ldcg(a.small_r + i);
                srid[i] = __ldcg(a.small_rid + i);
            }
            __syncthreads();
            block_sort(sr, srid, cnt);
            const uint64_t base = a.k - krem;
            for (uint64_t i = threadIdx.x; i < krem; i += TK_TPB) {
                a.out_r0[base + i] = sr[i];
                a.out_rid0[base + i] = srid[i];
            }
            __syncthreads();
        }
        if (a.k <= TK_SMALL) {
            const int cnt = static_cast<int>(a.k);
            for (int i = threadIdx.x; i < cnt; i += TK_TPB) {
                sr[i] = __ldcg(a.out_r0 + i);
                srid[i] = __ldcg(a.out_rid0 + i);
            }
            __syncthreads();
            block_sort(sr, srid, cnt);
            for (int i = threadIdx.x; i < cnt; i += TK_TPB) write_result(a, i, sr[i], srid[i]);
            if (threadIdx.x == 0 && a.dev_status) *a.dev_status = ld_volatile_i32(&ctl->err);
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
        block_sort(sr, srid, cnt);
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
    a.use_sample = p.use_sample;
    a.sample_rank = p.sample_rank;
}

int topk_grid(int device, int max_ctas_per_sm) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TK_SMEM) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_kernel, TK_TPB, TK_SMEM) !=
        cudaSuccess)
        return 0;
    per_sm = std::min(per_sm, max_ctas_per_sm);
    return sms * per_sm;
}

cudaError_t topk_launch(const TopkArgs& args, int grid, cudaStream_t stream) {
    void* params[] = {const_cast<TopkArgs*>(&args)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(topk_kernel), dim3(grid), dim3(TK_TPB),
                                       params, TK_SMEM, stream);
}

}  // namespace olap
