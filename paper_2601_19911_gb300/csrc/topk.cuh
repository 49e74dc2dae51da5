// Top-K selection (ORDER BY key LIMIT K, Sec. III-A) on the GPU: launch
// arguments and host entry of the cooperative select kernel.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace olap {

constexpr int TK_TPB = 512;               // threads per CTA
constexpr int TK_DIG = 12;                // default radix digit width (8..12; histograms hold 2^12 bins)
constexpr int TK_DIG_MIN = 8;
constexpr int TK_BINS = 1 << TK_DIG;
constexpr int TK_SMALL = 4096;            // entries one CTA sorts in shared memory
constexpr int TK_SAMPLE = 8192;           // sample size of the threshold estimate
constexpr int TK_SPT = TK_SAMPLE / TK_TPB;
constexpr int TK_PREP_CTAS = TK_SAMPLE / TK_TPB;   // prepare CTAs on the sampled path: one key per thread
constexpr int TK_UNROLL = 4;              // 16-byte loads in flight per thread (register filter)
constexpr uint64_t TK_DIRECT_N = 1ull << 21;   // at or below: no sample, refine the input
constexpr int TK_RANK_MAX = 8192;         // survivors ranked in shared memory by the whole grid
constexpr int TK_SORT_SMEM = TK_RANK_MAX * 12;  // select kernel shared bytes (ranking / sort tile / histogram)
constexpr int TK_MAX_STAGES = 16;         // full + empty mbarrier pairs reserved after the ring
constexpr int TK_SMEM_MAX = 227 * 1024;   // opt-in shared memory per CTA
// The streaming filter runs as its own kernel: 256-thread CTAs, several per
// SM, each with a ring of bulk copies (default 16 KB x 3, four CTAs per SM);
// the register-load flavour uses CTAs of 256, 512 (default) or 1024 threads.
constexpr int TKF_TPB = 256;
constexpr int TKR_TPB = 512;
constexpr int TK_TILE_DEFAULT = 16384;
constexpr int TK_STAGES_DEFAULT = 3;
constexpr int TK_CTAS_PER_SM_DEFAULT = 4;

// Filter flavours: 16-byte register loads, or bulk copies through a ring of
// shared-memory stages (the default).
enum TopkFilter { TK_FILTER_REGS = 0, TK_FILTER_BULK = 1 };

// Device control block, zeroed by CTA 0 at the start of every launch.
struct TopkCtl {
    unsigned long long cand_count;   // filter: rank words <= threshold seen
    unsigned long long thresh;       // sample threshold (inclusive)
    unsigned long long out_count;    // split: entries below the final prefix
    unsigned long long eq_count;     // split: prefix-equal entries taken wholesale
    unsigned long long small_count;  // split: prefix-equal entries kept for the finish
    int err;                         // olap_status of the device side
    int path;                        // 0 direct, 1 sampled candidates, 2 fallback
    int passes;                      // refine passes run
    int pad;
    // AND and OR of the composite words (w0, w1) of the entries a refine pass
    // saw (three slots, by pass), and of the selected entries before the
    // finish partition: {and0, and1, or0, or1}.  Bits where AND == OR are
    // common to all those entries.
    unsigned long long ao[3][4];
    unsigned long long fin[4];
    // %globaltimer stamps: prepare start, prepare end (sample done), select
    // start (filter done), source decided, refine done, split done, end,
    // small-buffer finish done, survivor sort done.
    unsigned long long ts[9];
};

struct TopkArgs {
    const void* keys;
    const uint32_t* rowids;          // NULL => row-id = index
    uint64_t n;
    uint64_t k;                      // already min(k, n), > 0
    int kind;                        // olap_key_type
    int w4;                          // 4-byte keys (float32, int32, uint32)
    int desc;
    int use_sample;
    unsigned sample_rank;            // 1-based rank of the threshold in the sample
    int filter;                      // TopkFilter
    int fuse;                        // the filter folds the select's first radix pass (set at launch)
    int digit;                       // radix digit width, TK_DIG_MIN..TK_DIG (0 => TK_DIG)
    int tile_bytes;                  // bulk-copy size (multiple of 16 * TK_TPB)
    int stages;                      // copies in flight per CTA (<= TK_MAX_STAGES)
    TopkCtl* ctl;
    GridBar* bar;
    unsigned* ghist;                 // 3 x TK_BINS
    uint64_t* cand_r;
    uint32_t* cand_rid;
    uint64_t cand_cap;
    uint64_t* small_r;               // TK_SMALL
    uint32_t* small_rid;
    uint64_t* out_r0;                // k entries (selected, then sorted)
    uint32_t* out_rid0;
    uint64_t* out_r1;                // k entries, merge ping-pong (k > TK_SMALL)
    uint32_t* out_rid1;
    uint64_t* samples;               // TK_SAMPLE rank words of the sample (sampled path)
    void* out_keys;                  // caller's outputs (device)
    uint32_t* out_rowids;
    // Two-column key (ORDER BY c0, c1): keys / kind / desc describe c0 and
    // these c1; both columns are 4-byte kinds and the rank word is c0's rank
    // in the upper 32 bits and c1's in the lower 32 (w4 = 0).
    int pair;
    int kind2;
    int desc2;
    const void* keys2;
    void* out_keys2;
    int32_t* dev_status;             // optional device status word
};

// Plan of one Top-K call: which path and how much scratch it needs.
struct TopkPlan {
    int use_sample;
    unsigned sample_rank;
    uint64_t cand_cap;
};
TopkPlan topk_plan(uint64_t n, uint64_t k);

// Bytes of device scratch a call with this plan needs (all buffers above).
size_t topk_scratch_bytes(const TopkPlan& p, uint64_t k);

// Carve the scratch buffers of `args` out of `base` (256-byte aligned pieces).
void topk_carve(TopkArgs& args, const TopkPlan& p, void* base);

// Launch geometry of one Top-K: the filter's copy ring (tile x stages), the
// filter grids and the cooperative select grid.
struct TopkGeom {
    int tile_bytes;
    int stages;
    int ctas_per_sm;       // filter CTAs per SM (cap)
    int smem_bytes;        // filter dynamic shared bytes: ring + mbarriers
    int grid;              // cooperative select kernel CTAs
    int grid_small;        // the same for a candidate-path select with k <= TK_SMALL (one CTA per SM)
    int filter_grid;       // bulk-copy filter CTAs
    int regs_grid;         // register-load filter CTAs
    int regs_tpb;          // register-load filter threads per CTA (256, 512, 1024)
};
// Fill in the geometry for the requested ring and register-filter block size
// on `device`; 0 values take the defaults.  Returns false if the ring does not
// fit, the block size is not one of 256/512/1024, or no CTA fits.
bool topk_geometry(int device, int tile_bytes, int stages, int ctas_per_sm, int regs_tpb, TopkGeom* out);

// Enqueue one Top-K: prepare (1 CTA, or TK_PREP_CTAS that load the sample),
// the streaming filter when the sampled path is taken, then the cooperative
// select kernel.  Returns the first CUDA
// launch error.
// ev (optional, 4 events): recorded before the prepare kernel and after the
// prepare, filter and select kernels (the filter pair is empty when the plan
// has no sample filter).
cudaError_t topk_launch(const TopkArgs& args, const TopkGeom& geom, cudaStream_t stream,
                        cudaEvent_t* ev = nullptr);

}  // namespace olap
