// Top-K selection (ORDER BY key LIMIT K, Sec. III-A) on the GPU: launch
// arguments and host entry of the cooperative select kernel.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace olap {

constexpr int TK_TPB = 512;               // threads per CTA
constexpr int TK_DIG = 12;                // radix digit width of the refine passes
constexpr int TK_BINS = 1 << TK_DIG;
constexpr int TK_SMALL = 4096;            // entries one CTA sorts in shared memory
constexpr int TK_SAMPLE = 8192;           // sample size of the threshold estimate
constexpr int TK_SPT = TK_SAMPLE / TK_TPB;
constexpr int TK_UNROLL = 4;              // 16-byte loads in flight per thread
constexpr uint64_t TK_DIRECT_N = 1ull << 21;   // at or below: no sample, refine the input
constexpr int TK_SMEM = TK_SMALL * 12;    // shared bytes: sort tile (or histogram)

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
};

struct TopkArgs {
    const void* keys;
    const uint32_t* rowids;          // NULL => row-id = index
    uint64_t n;
    uint64_t k;                      // already min(k, n), > 0
    int f32;
    int desc;
    int use_sample;
    unsigned sample_rank;            // 1-based rank of the threshold in the sample
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
    void* out_keys;                  // caller's outputs (device)
    uint32_t* out_rowids;
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

// CTAs of the cooperative grid on `device` (SMs x resident CTAs, capped).
int topk_grid(int device, int max_ctas_per_sm);

// Enqueue the cooperative kernel.  Returns the CUDA launch error.
cudaError_t topk_launch(const TopkArgs& args, int grid, cudaStream_t stream);

}  // namespace olap
