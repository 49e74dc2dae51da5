// Host-side context of the OLAP library: device, stream, device scratch
// arena, pinned staging buffers and the last error message.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <set>
#include <string>

#include "hostcopy.h"
#include "olap.h"
#include "topk.cuh"

// The context's small device area: [0] probe count word, [256] row queue
// counter, [1024] the probe's plan, [1536] the plan kernel's counters,
// [2048] the self-test words, [16384] the plan kernel's packed sample.
constexpr size_t OLAP_AUX_BYTES = 32768;

struct olap_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    olap_opts opts{};
    int sm_count = 0;
    olap::TopkGeom topk_geom{};       // Top-K launch geometry

    // Device scratch arena (grow-only).  Its first bytes hold the grid
    // barrier of the cooperative kernels, which must start zeroed.
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    bool barrier_dirty = false;       // a device wait expired: re-zero before use

    // Device copies of host inputs / outputs (grow-only).
    void* dev_in = nullptr;
    size_t dev_in_bytes = 0;
    void* dev_out = nullptr;
    size_t dev_out_bytes = 0;

    // Pinned double buffers for pageable host data, and their copy events.
    void* pinned[2] = {nullptr, nullptr};
    size_t pinned_bytes = 0;
    cudaEvent_t pinned_ev[2] = {nullptr, nullptr};
    olap::HostCopyPool* copy_pool = nullptr;   // host threads of the staging copies

    // Small pinned words for device status read-back, and a small device
    // area for counters of blocking calls (4 KiB).
    int32_t* host_status = nullptr;
    void* aux = nullptr;               // small device area (OLAP_AUX_BYTES): counters, the probe's plan and sample

    // Control block of the last Top-K launched (diagnostics).
    void* last_topk_ctl = nullptr;

    // Kernels launched for this context (a batch replay counts its graph's
    // kernels).
    uint64_t launches = 0;

    // Optional per-kernel timing: events around the kernels of the last Top-K
    // (4) and of the last join probe (2) launched while timing is on.
    bool time_kernels = false;
    cudaEvent_t kev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool topk_timed = false, probe_timed = false, topk_filtered = false;

    // Full-row offload scratch (grow-only): the extracted key column, the
    // selection's outputs and the gathered rows.
    void* rows_buf = nullptr;
    size_t rows_buf_bytes = 0;

    // Partitioned-probe scratch (grow-only): partitioned keys, row-ids and
    // the per-CTA partition counts.
    void* part = nullptr;
    size_t part_bytes = 0;
    uint64_t l2_bytes = 0;            // device L2 size
    bool host_direct = false;         // copy pageable host memory with a kernel (no CPU staging)

    // The last probe enqueued: partitions, rows, and its pre-probe control
    // block on the device (NULL when it ran none).
    int last_probe_parts = 0;
    uint64_t last_probe_n = 0;
    const void* last_probe_pf = nullptr;
    bool last_rowids_in_place = false;   // the last blocking Top-K read its row-ids in host memory

    // Device memory held by live join tables built through this context.
    uint64_t table_bytes = 0;
    std::set<olap_join_table*> tables;

    std::string last_error;
};

namespace olap {

// Record an error message on the context and return the status.
olap_status fail(olap_ctx* ctx, olap_status st, const std::string& msg);
// Map a CUDA error to OLAP_E_CUDA with the call site in the message.
olap_status cuda_fail(olap_ctx* ctx, cudaError_t e, const char* what);

// Grow-only device buffers of the context.
olap_status ensure_scratch(olap_ctx* ctx, size_t bytes);
olap_status ensure_dev_in(olap_ctx* ctx, size_t bytes);
olap_status ensure_dev_out(olap_ctx* ctx, size_t bytes);
olap_status ensure_pinned(olap_ctx* ctx);
olap_status ensure_part(olap_ctx* ctx, size_t bytes);

// Partitions a probe of n rows against table t uses (1 = direct probe), and
// the partition scratch it needs (0 for a direct probe).
int probe_parts(const olap_ctx* ctx, const olap_join_table* t, uint64_t n);
size_t probe_scratch_bytes(const olap_ctx* ctx, const olap_join_table* t, uint64_t n);

// Copy `bytes` from host memory of kind `where` to device `dst` on the
// context stream; pageable memory goes through the pinned double buffers.
olap_status copy_h2d(olap_ctx* ctx, void* dst, const void* src, size_t bytes, olap_mem where);
// Copy device `src` to host memory of kind `where` (pageable through pinned).
olap_status copy_d2h(olap_ctx* ctx, void* dst, const void* src, size_t bytes, olap_mem where);

// Bytes of device memory the context may still allocate under its budget.
bool within_budget(const olap_ctx* ctx, size_t extra);

// Row-store helpers (full-row offload): pull the key field out of n rows
// into a dense column; gather k rows by index.  Enqueue only.
cudaError_t rows_extract(const void* rows, uint64_t n, uint32_t row_bytes, uint32_t key_offset, int key_width,
                         void* keys, int grid, cudaStream_t s);
cudaError_t rows_gather(const void* rows, uint32_t row_bytes, const uint32_t* idx, uint64_t k, void* out, int grid,
                        cudaStream_t s);

}  // namespace olap
