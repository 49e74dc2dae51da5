// C ABI of the OLAP library: contexts, memory movement of the key-only
// contract (Sec. II-C: only (key, row-id) crosses the link, only row pointers
// come back) and the Top-K entry points.
#include <algorithm>
#include <cstring>
#include <string>

#include "ctx.h"
#include "topk.cuh"

// Join tables outlive nothing: a context being destroyed forgets the tables it
// built (they stay valid and are freed with olap_join_free).
void detach_tables(olap_ctx* ctx);

namespace olap {

olap_status fail(olap_ctx* ctx, olap_status st, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

olap_status cuda_fail(olap_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(ctx, OLAP_E_NOMEM, m);
    return fail(ctx, OLAP_E_CUDA, m);
}

bool within_budget(const olap_ctx* ctx, size_t extra) {
    if (ctx->opts.mem_budget_bytes == 0) return true;
    const uint64_t held = ctx->scratch_bytes + ctx->dev_in_bytes + ctx->dev_out_bytes + ctx->table_bytes;
    return held + extra <= ctx->opts.mem_budget_bytes;
}

static olap_status grow(olap_ctx* ctx, void** buf, size_t* have, size_t need, const char* what) {
    if (*have >= need) return OLAP_OK;
    size_t want = std::max(need, *have + *have / 2);
    want = (want + 0xFFFFF) & ~static_cast<size_t>(0xFFFFF);
    if (!within_budget(ctx, want - *have))
        return fail(ctx, OLAP_E_NOMEM, std::string(what) + ": device memory budget exceeded");
    // Work on any stream may still use the old buffer.
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    e = cudaMalloc(buf, want);
    if (e != cudaSuccess) {
        *buf = nullptr;
        cudaGetLastError();
        return cuda_fail(ctx, e, what);
    }
    *have = want;
    return OLAP_OK;
}

olap_status ensure_scratch(olap_ctx* ctx, size_t bytes) {
    const bool fresh = ctx->scratch_bytes < bytes;
    olap_status st = grow(ctx, &ctx->scratch, &ctx->scratch_bytes, bytes, "scratch allocation");
    if (st != OLAP_OK) return st;
    if (fresh || ctx->barrier_dirty) {
        cudaError_t e = cudaMemsetAsync(ctx->scratch, 0, 256, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "barrier reset");
        ctx->barrier_dirty = false;
    }
    return OLAP_OK;
}

olap_status ensure_dev_in(olap_ctx* ctx, size_t bytes) {
    return grow(ctx, &ctx->dev_in, &ctx->dev_in_bytes, bytes, "input staging allocation");
}

olap_status ensure_dev_out(olap_ctx* ctx, size_t bytes) {
    return grow(ctx, &ctx->dev_out, &ctx->dev_out_bytes, bytes, "output staging allocation");
}

static olap_status grow_rows_buf(olap_ctx* ctx, size_t bytes) {
    return grow(ctx, &ctx->rows_buf, &ctx->rows_buf_bytes, bytes, "full-row scratch allocation");
}

olap_status ensure_part(olap_ctx* ctx, size_t bytes) {
    return grow(ctx, &ctx->part, &ctx->part_bytes, bytes, "probe partition allocation");
}

olap_status ensure_pinned(olap_ctx* ctx) {
    if (ctx->pinned_bytes) return OLAP_OK;
    const size_t b = ctx->opts.staging_bytes ? ctx->opts.staging_bytes : (64ull << 20);
    // All or nothing: a partial set (one buffer, or a buffer without its
    // event) would make the staged copies spin on zero-length chunks.
    auto undo = [&](cudaError_t e, const char* what) {
        cudaGetLastError();
        for (int i = 0; i < 2; ++i) {
            if (ctx->pinned[i]) cudaFreeHost(ctx->pinned[i]);
            if (ctx->pinned_ev[i]) cudaEventDestroy(ctx->pinned_ev[i]);
            ctx->pinned[i] = nullptr;
            ctx->pinned_ev[i] = nullptr;
        }
        return cuda_fail(ctx, e, what);
    };
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaMallocHost(&ctx->pinned[i], b);
        if (e != cudaSuccess) {
            ctx->pinned[i] = nullptr;
            return undo(e, "pinned staging allocation");
        }
        e = cudaEventCreateWithFlags(&ctx->pinned_ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            ctx->pinned_ev[i] = nullptr;
            return undo(e, "staging event");
        }
    }
    ctx->pinned_bytes = b;
    if (!ctx->copy_pool) {
        const int threads = ctx->opts.staging_threads ? ctx->opts.staging_threads : 4;
        ctx->copy_pool = new HostCopyPool(threads - 1);
    }
    return OLAP_OK;
}

// Copy between pageable host memory and device memory by a kernel that
// dereferences the host addresses itself.  Used only when the device reads
// and writes pageable memory coherently through the host's page tables
// (Grace systems over NVLink-C2C), so no staging copy on the CPU is needed.
// U is the widest access size with which source and destination line up.
template <typename T>
__global__ void __launch_bounds__(256) direct_copy_kernel(unsigned char* dst, const unsigned char* src, size_t head,
                                                          size_t units, size_t tail) {
    const size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = t; i < head; i += stride) dst[i] = src[i];
    const T* s = reinterpret_cast<const T*>(src + head);
    T* d = reinterpret_cast<T*>(dst + head);
    for (size_t i = t; i < units; i += stride) d[i] = s[i];
    const size_t base = head + units * sizeof(T);
    for (size_t i = t; i < tail; i += stride) dst[base + i] = src[base + i];
}

static olap_status direct_copy(olap_ctx* ctx, void* dst, const void* src, size_t bytes, const char* what) {
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst), s = reinterpret_cast<uintptr_t>(src);
    size_t u = 16;
    while (u > 1 && ((d ^ s) & (u - 1))) u >>= 1;
    const size_t head = std::min(bytes, static_cast<size_t>((u - (d & (u - 1))) & (u - 1)));
    const size_t units = (bytes - head) / u;
    const size_t tail = bytes - head - units * u;
    const unsigned grid = static_cast<unsigned>(ctx->sm_count * 4);
    unsigned char* dp = static_cast<unsigned char*>(dst);
    const unsigned char* sp = static_cast<const unsigned char*>(src);
    if (u == 16) direct_copy_kernel<uint4><<<grid, 256, 0, ctx->stream>>>(dp, sp, head, units, tail);
    else if (u == 8) direct_copy_kernel<uint64_t><<<grid, 256, 0, ctx->stream>>>(dp, sp, head, units, tail);
    else if (u == 4) direct_copy_kernel<uint32_t><<<grid, 256, 0, ctx->stream>>>(dp, sp, head, units, tail);
    else if (u == 2) direct_copy_kernel<uint16_t><<<grid, 256, 0, ctx->stream>>>(dp, sp, head, units, tail);
    else direct_copy_kernel<uint8_t><<<grid, 256, 0, ctx->stream>>>(dp, sp, head, units, tail);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    ctx->launches += 1;
    return OLAP_OK;
}

// Self-test of the bounded device waits: one thread waits, with the wait
// the grid barriers use, on a word that nothing writes.
__global__ void wait_selftest_kernel(const unsigned* word, int* err, long long limit) {
    if (threadIdx.x == 0 && blockIdx.x == 0) wait_changed(word, 0u, err, limit);
}

olap_status copy_h2d(olap_ctx* ctx, void* dst, const void* src, size_t bytes, olap_mem where) {
    if (bytes == 0) return OLAP_OK;
    cudaError_t e;
    if (where == OLAP_MEM_HOST && ctx->host_direct) return direct_copy(ctx, dst, src, bytes, "direct H2D copy");
    if (where == OLAP_MEM_DEVICE) {
        e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        return e == cudaSuccess ? OLAP_OK : cuda_fail(ctx, e, "device copy");
    }
    if (where == OLAP_MEM_HOST_PINNED) {
        e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
        return e == cudaSuccess ? OLAP_OK : cuda_fail(ctx, e, "pinned H2D copy");
    }
    // Pageable: host memcpy into one pinned buffer while the other one's DMA runs.
    olap_status st = ensure_pinned(ctx);
    if (st != OLAP_OK) return st;
    const unsigned char* s = static_cast<const unsigned char*>(src);
    unsigned char* d = static_cast<unsigned char*>(dst);
    size_t off = 0;
    int slot = 0;
    while (off < bytes) {
        const size_t len = std::min(ctx->pinned_bytes, bytes - off);
        e = cudaEventSynchronize(ctx->pinned_ev[slot]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "staging wait");
        ctx->copy_pool->copy(ctx->pinned[slot], s + off, len);
        e = cudaMemcpyAsync(d + off, ctx->pinned[slot], len, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "staged H2D copy");
        e = cudaEventRecord(ctx->pinned_ev[slot], ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "staging event record");
        off += len;
        slot ^= 1;
    }
    return OLAP_OK;
}

olap_status copy_d2h(olap_ctx* ctx, void* dst, const void* src, size_t bytes, olap_mem where) {
    if (bytes == 0) return OLAP_OK;
    cudaError_t e;
    if (where == OLAP_MEM_DEVICE) {
        e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        return e == cudaSuccess ? OLAP_OK : cuda_fail(ctx, e, "device copy");
    }
    if (where == OLAP_MEM_HOST_PINNED) {
        e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
        return e == cudaSuccess ? OLAP_OK : cuda_fail(ctx, e, "pinned D2H copy");
    }
    if (ctx->host_direct) return direct_copy(ctx, dst, src, bytes, "direct D2H copy");
    olap_status st = ensure_pinned(ctx);
    if (st != OLAP_OK) return st;
    const unsigned char* s = static_cast<const unsigned char*>(src);
    unsigned char* d = static_cast<unsigned char*>(dst);
    // Chunks alternate between the two pinned buffers; the host copies chunk
    // i out of its buffer once that buffer's DMA has finished, while the DMA
    // of chunk i+1 runs into the other buffer.
    size_t off = 0, pend_off = 0, pend_len = 0;
    int slot = 0, pend_slot = -1;
    while (off < bytes || pend_slot >= 0) {
        if (off < bytes) {
            const size_t len = std::min(ctx->pinned_bytes, bytes - off);
            e = cudaMemcpyAsync(ctx->pinned[slot], s + off, len, cudaMemcpyDeviceToHost, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "staged D2H copy");
            e = cudaEventRecord(ctx->pinned_ev[slot], ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "staging event record");
            if (pend_slot >= 0) {
                e = cudaEventSynchronize(ctx->pinned_ev[pend_slot]);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "staging wait");
                ctx->copy_pool->copy(d + pend_off, ctx->pinned[pend_slot], pend_len);
            }
            pend_slot = slot;
            pend_off = off;
            pend_len = len;
            off += len;
            slot ^= 1;
        } else {
            e = cudaEventSynchronize(ctx->pinned_ev[pend_slot]);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "staging wait");
            ctx->copy_pool->copy(d + pend_off, ctx->pinned[pend_slot], pend_len);
            pend_slot = -1;
        }
    }
    return OLAP_OK;
}

// The second column of a two-column key (ORDER BY c0, c1).
struct PairSpec {
    const void* keys;
    olap_key_type type;
    olap_order order;
    void* out_keys;
};

// Enqueue one Top-K on device pointers.  The caller has validated arguments.
static olap_status topk_enqueue(olap_ctx* ctx, const void* d_keys, olap_key_type type,
                                const uint32_t* d_rowids, uint64_t n, uint64_t kk, olap_order order,
                                void* d_out_keys, uint32_t* d_out_rowids, int32_t* dev_status,
                                cudaStream_t stream, TopkCtl** ctl_out, const PairSpec* pair = nullptr) {
    const TopkPlan plan = topk_plan(n, kk);
    const bool reset = ctx->barrier_dirty || ctx->scratch_bytes < topk_scratch_bytes(plan, kk);
    olap_status st = ensure_scratch(ctx, topk_scratch_bytes(plan, kk));
    if (st != OLAP_OK) return st;
    if (reset && stream != ctx->stream) {
        // The barrier reset ran on the context stream; order the launch after it.
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "barrier reset wait");
    }
    TopkArgs a{};
    a.keys = d_keys;
    a.rowids = d_rowids;
    a.n = n;
    a.k = kk;
    a.kind = type;
    a.w4 = key_bytes(type) == 4;
    a.desc = order == OLAP_DESC;
    topk_carve(a, plan, ctx->scratch);
    a.out_keys = d_out_keys;
    a.out_rowids = d_out_rowids;
    a.dev_status = dev_status;
    if (pair) {
        a.pair = 1;
        a.w4 = 0;                                           // 64-bit composite rank words
        a.keys2 = pair->keys;
        a.kind2 = pair->type;
        a.desc2 = pair->order == OLAP_DESC;
        a.out_keys2 = pair->out_keys;
    }
    a.filter = ctx->opts.topk_filter == OLAP_FILTER_BULK ? TK_FILTER_BULK : TK_FILTER_REGS;
    a.digit = ctx->opts.topk_digit_bits ? ctx->opts.topk_digit_bits : TK_DIG;
    ctx->last_topk_ctl = a.ctl;
    ctx->last_rowids_in_place = false;      // olap_topk sets it after this when it applies
    ctx->topk_timed = ctx->time_kernels;
    ctx->topk_filtered = plan.use_sample;
    cudaError_t e = topk_launch(a, ctx->topk_geom, stream, ctx->time_kernels ? ctx->kev : nullptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "Top-K launch");
    }
    ctx->launches += plan.use_sample ? 3 : 2;           // prepare, [filter,] select
    if (ctl_out) *ctl_out = a.ctl;
    return OLAP_OK;
}

static olap_status check_topk_args(olap_ctx* ctx, const void* keys, olap_key_type type, uint64_t n,
                                   uint64_t kk, olap_order order, const void* out_keys,
                                   const void* out_rowids) {
    if (type < OLAP_KEY_I64 || type > OLAP_KEY_U32) return fail(ctx, OLAP_E_INVALID, "bad key type");
    if (order != OLAP_ASC && order != OLAP_DESC) return fail(ctx, OLAP_E_INVALID, "bad order");
    if (n >= (1ull << 32)) return fail(ctx, OLAP_E_INVALID, "n must be below 2^32");
    if (n && !keys) return fail(ctx, OLAP_E_INVALID, "keys is NULL");
    if (kk && (!out_keys || !out_rowids)) return fail(ctx, OLAP_E_INVALID, "output pointer is NULL");
    const size_t w = key_bytes(type);
    if (reinterpret_cast<uintptr_t>(keys) % w) return fail(ctx, OLAP_E_INVALID, "keys misaligned");
    return OLAP_OK;
}

}  // namespace olap

using namespace olap;

extern "C" {

olap_status olap_ctx_create(const olap_opts* opts, olap_ctx** out) {
    if (!out) return OLAP_E_INVALID;
    *out = nullptr;
    olap_ctx* ctx = new olap_ctx();
    if (opts) ctx->opts = *opts;
    const int jp = ctx->opts.join_partitions;
    if (ctx->opts.load_factor < 0.0 || ctx->opts.load_factor > 0.9 || ctx->opts.topk_filter < 0 ||
        ctx->opts.topk_filter > OLAP_FILTER_REGS || jp < 0 || jp > 256 || (jp > 1 && (jp & (jp - 1))) ||
        ctx->opts.join_bucket_loads < OLAP_LOADS_AUTO || ctx->opts.join_bucket_loads > OLAP_LOADS_L2_ONLY ||
        (ctx->opts.topk_digit_bits != 0 && (ctx->opts.topk_digit_bits < 8 || ctx->opts.topk_digit_bits > 12)) ||
        ctx->opts.host_access < OLAP_HOST_AUTO || ctx->opts.host_access > OLAP_HOST_STAGED ||
        ctx->opts.batch_overlap < 0 || ctx->opts.batch_overlap > 1 || ctx->opts.batch_topk_ctas_per_sm < 0 ||
        ctx->opts.batch_topk_ctas_per_sm > 2 || ctx->opts.join_prefilter < OLAP_PREFILTER_AUTO ||
        ctx->opts.join_prefilter > OLAP_PREFILTER_ON || ctx->opts.staging_threads < 0 ||
        ctx->opts.staging_threads > 64 ||
        (ctx->opts.block_threads != 0 && ctx->opts.block_threads != 256 && ctx->opts.block_threads != 512 &&
         ctx->opts.block_threads != 1024) ||
        (ctx->opts.l2_fetch_bytes != 0 && ctx->opts.l2_fetch_bytes != 32 && ctx->opts.l2_fetch_bytes != 64 &&
         ctx->opts.l2_fetch_bytes != 128)) {
        delete ctx;
        return OLAP_E_INVALID;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev <= ctx->opts.device || ctx->opts.device < 0) {
        cudaGetLastError();
        delete ctx;
        return OLAP_E_CUDA;
    }
    ctx->device = ctx->opts.device;
    auto bail = [&](cudaError_t) {
        cudaGetLastError();
        olap_ctx_destroy(ctx);
        return OLAP_E_CUDA;
    };
    if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return bail(e);
    if (ctx->opts.stream) {
        ctx->stream = static_cast<cudaStream_t>(ctx->opts.stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
        ctx->own_stream = true;
    }
    if ((e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess)
        return bail(e);
    int l2 = 0;
    if ((e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device)) != cudaSuccess) return bail(e);
    ctx->l2_bytes = static_cast<uint64_t>(l2);
    int pageable = 0, host_pt = 0;
    if ((e = cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, ctx->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&host_pt, cudaDevAttrPageableMemoryAccessUsesHostPageTables, ctx->device)) !=
            cudaSuccess)
        return bail(e);
    ctx->host_direct = ctx->opts.host_access != OLAP_HOST_STAGED && pageable && host_pt;
    if (ctx->opts.l2_fetch_bytes &&
        (e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, static_cast<size_t>(ctx->opts.l2_fetch_bytes))) !=
            cudaSuccess)
        return bail(e);
    TopkGeom g;
    if (!topk_geometry(ctx->device, ctx->opts.topk_tile_bytes, ctx->opts.topk_stages,
                       ctx->opts.topk_ctas_per_sm, ctx->opts.block_threads, &g)) {
        cudaGetLastError();
        olap_ctx_destroy(ctx);
        return OLAP_E_INVALID;
    }
    ctx->topk_geom = g;
    if ((e = cudaMallocHost(reinterpret_cast<void**>(&ctx->host_status), 64)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&ctx->aux, OLAP_AUX_BYTES)) != cudaSuccess) return bail(e);
    if ((e = cudaMemset(ctx->aux, 0, OLAP_AUX_BYTES)) != cudaSuccess) return bail(e);
    *out = ctx;
    return OLAP_OK;
}

void olap_ctx_destroy(olap_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->dev_in) cudaFree(ctx->dev_in);
    if (ctx->dev_out) cudaFree(ctx->dev_out);
    if (ctx->part) cudaFree(ctx->part);
    if (ctx->rows_buf) cudaFree(ctx->rows_buf);
    for (int i = 0; i < 2; ++i) {
        if (ctx->pinned[i]) cudaFreeHost(ctx->pinned[i]);
        if (ctx->pinned_ev[i]) cudaEventDestroy(ctx->pinned_ev[i]);
    }
    delete ctx->copy_pool;
    for (cudaEvent_t ev : ctx->kev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->host_status) cudaFreeHost(ctx->host_status);
    if (ctx->aux) cudaFree(ctx->aux);
    detach_tables(ctx);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* olap_last_error(const olap_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

void* olap_ctx_stream(const olap_ctx* ctx) { return ctx ? static_cast<void*>(ctx->stream) : nullptr; }

int olap_ctx_host_direct(const olap_ctx* ctx) { return ctx && ctx->host_direct ? 1 : 0; }

olap_status olap_selftest_wait(olap_ctx* ctx, uint64_t limit_cycles, int32_t* out_status) {
    if (!ctx || !out_status) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (limit_cycles == 0 || limit_cycles > (1ull << 31)) return fail(ctx, OLAP_E_INVALID, "limit out of range");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");
    // aux: [word nobody writes][status], in the context's small device area
    unsigned* word = static_cast<unsigned*>(ctx->aux) + 512;
    int* err = reinterpret_cast<int*>(static_cast<unsigned*>(ctx->aux) + 520);
    if ((e = cudaMemsetAsync(word, 0, 64, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "self-test reset");
    wait_selftest_kernel<<<1, 32, 0, ctx->stream>>>(word, err, static_cast<long long>(limit_cycles));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "self-test launch");
    ctx->launches += 1;
    if ((e = cudaMemcpyAsync(ctx->host_status, err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "self-test wait");
    *out_status = *ctx->host_status;
    return OLAP_OK;
}

olap_status olap_ctx_sync(olap_ctx* ctx) {
    if (!ctx) return OLAP_E_INVALID;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? OLAP_OK : cuda_fail(ctx, e, "stream synchronize");
}

olap_status olap_topk_rows(olap_ctx* ctx, const void* rows, olap_mem in_where, uint64_t n, uint32_t row_bytes,
                           uint32_t key_offset, olap_key_type type, uint64_t k, olap_order order, void* out_rows,
                           uint32_t* out_rowids, olap_mem out_where, uint64_t* out_count) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!out_count) return fail(ctx, OLAP_E_INVALID, "out_count is NULL");
    *out_count = 0;
    if (in_where < OLAP_MEM_HOST || in_where > OLAP_MEM_DEVICE || out_where < OLAP_MEM_HOST ||
        out_where > OLAP_MEM_DEVICE)
        return fail(ctx, OLAP_E_INVALID, "bad memory kind");
    if (type < OLAP_KEY_I64 || type > OLAP_KEY_U32) return fail(ctx, OLAP_E_INVALID, "bad key type");
    if (order != OLAP_ASC && order != OLAP_DESC) return fail(ctx, OLAP_E_INVALID, "bad order");
    const size_t w = key_bytes(type);
    if (row_bytes == 0 || static_cast<uint64_t>(key_offset) + w > row_bytes)
        return fail(ctx, OLAP_E_INVALID, "key field outside the row");
    if (n >= (1ull << 32)) return fail(ctx, OLAP_E_INVALID, "n must be below 2^32");
    if (n && !rows) return fail(ctx, OLAP_E_INVALID, "rows is NULL");
    const uint64_t kk = std::min(k, n);
    if (kk && !out_rows) return fail(ctx, OLAP_E_INVALID, "out_rows is NULL");
    if (kk == 0) return OLAP_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");
    const uint64_t tbytes = n * row_bytes;
    const void* dr = rows;
    olap_status st;
    if (in_where != OLAP_MEM_DEVICE) {                      // the whole rows cross the link
        if ((st = ensure_dev_in(ctx, tbytes)) != OLAP_OK) return st;
        if ((st = copy_h2d(ctx, ctx->dev_in, rows, tbytes, in_where)) != OLAP_OK) return st;
        dr = ctx->dev_in;
    }
    // scratch: key column | selected keys | selected row-ids | gathered rows
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    const size_t o_keys = 0, o_sel = al(n * w), o_rid = o_sel + al(kk * w), o_rows = o_rid + al(kk * 4);
    if ((st = grow_rows_buf(ctx, o_rows + al(kk * row_bytes))) != OLAP_OK) return st;
    unsigned char* b = static_cast<unsigned char*>(ctx->rows_buf);
    const int grid = ctx->sm_count * 4;
    if ((e = rows_extract(dr, n, row_bytes, key_offset, static_cast<int>(w), b + o_keys, grid, ctx->stream)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "key extraction");
    ctx->launches += 1;
    TopkCtl* ctl = nullptr;
    uint32_t* drid = reinterpret_cast<uint32_t*>(b + o_rid);
    if ((st = topk_enqueue(ctx, b + o_keys, type, nullptr, n, kk, order, b + o_sel, drid, nullptr, ctx->stream,
                           &ctl)) != OLAP_OK)
        return st;
    if ((e = rows_gather(dr, row_bytes, drid, kk, b + o_rows, grid, ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "row gather");
    ctx->launches += 1;
    e = cudaMemcpyAsync(ctx->host_status, &ctl->err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read-back");
    if ((st = copy_d2h(ctx, out_rows, b + o_rows, kk * row_bytes, out_where)) != OLAP_OK) return st;
    if (out_rowids && (st = copy_d2h(ctx, out_rowids, drid, kk * 4, out_where)) != OLAP_OK) return st;
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return cuda_fail(ctx, e, "full-row Top-K");
    if (*ctx->host_status != OLAP_OK) {
        ctx->barrier_dirty = true;
        return fail(ctx, static_cast<olap_status>(*ctx->host_status), "Top-K device wait expired");
    }
    *out_count = kk;
    return OLAP_OK;
}

// On the sampled path only the candidates' row-ids are ever read (as the
// filter stages them), so row-ids in page-locked host memory can stay there:
// the kernels read those few in place over the host link (NVLink-C2C), and
// the copy carries the keys alone.  True, with *dr set to the row-ids'
// device-accessible address, when that applies.
static bool rowids_in_host(const uint32_t* rowids, olap_mem where, uint64_t n, uint64_t kk, const uint32_t** dr) {
    if (!rowids || where != OLAP_MEM_HOST_PINNED || !topk_plan(n, kk).use_sample) return false;
    void* mapped = nullptr;
    if (cudaHostGetDevicePointer(&mapped, const_cast<uint32_t*>(rowids), 0) != cudaSuccess || !mapped) {
        cudaGetLastError();
        return false;
    }
    *dr = static_cast<const uint32_t*>(mapped);
    return true;
}

olap_status olap_topk(olap_ctx* ctx, const void* keys, olap_key_type type, const uint32_t* rowids,
                      olap_mem in_where, uint64_t n, uint64_t k, olap_order order, void* out_keys,
                      uint32_t* out_rowids, olap_mem out_where, uint64_t* out_count) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!out_count) return fail(ctx, OLAP_E_INVALID, "out_count is NULL");
    *out_count = 0;
    if (in_where < OLAP_MEM_HOST || in_where > OLAP_MEM_DEVICE || out_where < OLAP_MEM_HOST ||
        out_where > OLAP_MEM_DEVICE)
        return fail(ctx, OLAP_E_INVALID, "bad memory kind");
    const uint64_t kk = std::min(k, n);
    olap_status st = check_topk_args(ctx, keys, type, n, kk, order, out_keys, out_rowids);
    if (st != OLAP_OK) return st;
    if (kk == 0) return OLAP_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");
    const size_t w = key_bytes(type);

    // Key-only input: keys (and explicit row-ids) to the device; pinned
    // row-ids on the sampled path stay where they are (rowids_in_host).
    const void* dk = keys;
    const uint32_t* dr = rowids;
    const bool rowids_in_place = rowids_in_host(rowids, in_where, n, kk, &dr);
    if (in_where != OLAP_MEM_DEVICE) {
        const size_t kbytes = (n * w + 255) & ~static_cast<size_t>(255);
        const bool copy_rowids = rowids && !rowids_in_place;
        st = ensure_dev_in(ctx, kbytes + (copy_rowids ? n * 4 : 0));
        if (st != OLAP_OK) return st;
        st = copy_h2d(ctx, ctx->dev_in, keys, n * w, in_where);
        if (st != OLAP_OK) return st;
        dk = ctx->dev_in;
        if (copy_rowids) {
            dr = reinterpret_cast<const uint32_t*>(static_cast<unsigned char*>(ctx->dev_in) + kbytes);
            st = copy_h2d(ctx, const_cast<uint32_t*>(dr), rowids, n * 4, in_where);
            if (st != OLAP_OK) return st;
        }
    }

    void* dok = out_keys;
    uint32_t* dor = out_rowids;
    const size_t okb = (kk * w + 255) & ~static_cast<size_t>(255);
    if (out_where != OLAP_MEM_DEVICE) {
        st = ensure_dev_out(ctx, okb + kk * 4);
        if (st != OLAP_OK) return st;
        dok = ctx->dev_out;
        dor = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ctx->dev_out) + okb);
    }
    TopkCtl* ctl = nullptr;
    st = topk_enqueue(ctx, dk, type, dr, n, kk, order, dok, dor, nullptr, ctx->stream, &ctl);
    if (st != OLAP_OK) return st;
    ctx->last_rowids_in_place = rowids_in_place;
    e = cudaMemcpyAsync(ctx->host_status, &ctl->err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read-back");
    if (out_where != OLAP_MEM_DEVICE) {
        st = copy_d2h(ctx, out_keys, dok, kk * w, out_where);
        if (st != OLAP_OK) return st;
        st = copy_d2h(ctx, out_rowids, dor, kk * 4, out_where);
        if (st != OLAP_OK) return st;
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "Top-K");
    if (*ctx->host_status != OLAP_OK) {
        ctx->barrier_dirty = true;
        return fail(ctx, static_cast<olap_status>(*ctx->host_status), "Top-K device wait expired");
    }
    *out_count = kk;
    return OLAP_OK;
}

olap_status olap_topk_pair(olap_ctx* ctx, const void* keys0, olap_key_type type0, olap_order order0,
                           const void* keys1, olap_key_type type1, olap_order order1, const uint32_t* rowids,
                           olap_mem in_where, uint64_t n, uint64_t k, void* out_keys0, void* out_keys1,
                           uint32_t* out_rowids, olap_mem out_where, uint64_t* out_count) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!out_count) return fail(ctx, OLAP_E_INVALID, "out_count is NULL");
    *out_count = 0;
    if (in_where < OLAP_MEM_HOST || in_where > OLAP_MEM_DEVICE || out_where < OLAP_MEM_HOST ||
        out_where > OLAP_MEM_DEVICE)
        return fail(ctx, OLAP_E_INVALID, "bad memory kind");
    const uint64_t kk = std::min(k, n);
    olap_status st = check_topk_args(ctx, keys0, type0, n, kk, order0, out_keys0, out_rowids);
    if (st != OLAP_OK) return st;
    if ((st = check_topk_args(ctx, keys1, type1, n, kk, order1, out_keys1, out_rowids)) != OLAP_OK) return st;
    if (key_bytes(type0) != 4 || key_bytes(type1) != 4)
        return fail(ctx, OLAP_E_UNIMPLEMENTED, "two-column keys take 4-byte columns (int32, uint32, float32)");
    if (kk == 0) return OLAP_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");

    // Key-only input: both key columns (and explicit row-ids) to the device;
    // pinned row-ids on the sampled path stay where they are.
    const void* d0 = keys0;
    const void* d1 = keys1;
    const uint32_t* dr = rowids;
    const bool rowids_in_place = rowids_in_host(rowids, in_where, n, kk, &dr);
    const size_t cb = (n * 4 + 255) & ~static_cast<size_t>(255);
    if (in_where != OLAP_MEM_DEVICE) {
        const bool copy_rowids = rowids && !rowids_in_place;
        if ((st = ensure_dev_in(ctx, 2 * cb + (copy_rowids ? n * 4 : 0))) != OLAP_OK) return st;
        unsigned char* m = static_cast<unsigned char*>(ctx->dev_in);
        if ((st = copy_h2d(ctx, m, keys0, n * 4, in_where)) != OLAP_OK) return st;
        if ((st = copy_h2d(ctx, m + cb, keys1, n * 4, in_where)) != OLAP_OK) return st;
        d0 = m;
        d1 = m + cb;
        if (copy_rowids) {
            dr = reinterpret_cast<const uint32_t*>(m + 2 * cb);
            if ((st = copy_h2d(ctx, const_cast<uint32_t*>(dr), rowids, n * 4, in_where)) != OLAP_OK) return st;
        }
    }
    void* do0 = out_keys0;
    void* do1 = out_keys1;
    uint32_t* dor = out_rowids;
    const size_t ob = (kk * 4 + 255) & ~static_cast<size_t>(255);
    if (out_where != OLAP_MEM_DEVICE) {
        if ((st = ensure_dev_out(ctx, 3 * ob)) != OLAP_OK) return st;
        unsigned char* m = static_cast<unsigned char*>(ctx->dev_out);
        do0 = m;
        do1 = m + ob;
        dor = reinterpret_cast<uint32_t*>(m + 2 * ob);
    }
    TopkCtl* ctl = nullptr;
    const PairSpec ps{d1, type1, order1, do1};
    if ((st = topk_enqueue(ctx, d0, type0, dr, n, kk, order0, do0, dor, nullptr, ctx->stream, &ctl, &ps)) !=
        OLAP_OK)
        return st;
    ctx->last_rowids_in_place = rowids_in_place;
    e = cudaMemcpyAsync(ctx->host_status, &ctl->err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read-back");
    if (out_where != OLAP_MEM_DEVICE) {
        if ((st = copy_d2h(ctx, out_keys0, do0, kk * 4, out_where)) != OLAP_OK) return st;
        if ((st = copy_d2h(ctx, out_keys1, do1, kk * 4, out_where)) != OLAP_OK) return st;
        if ((st = copy_d2h(ctx, out_rowids, dor, kk * 4, out_where)) != OLAP_OK) return st;
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "Top-K");
    if (*ctx->host_status != OLAP_OK) {
        ctx->barrier_dirty = true;
        return fail(ctx, static_cast<olap_status>(*ctx->host_status), "Top-K device wait expired");
    }
    *out_count = kk;
    return OLAP_OK;
}

olap_status olap_topk_async(olap_ctx* ctx, const void* d_keys, olap_key_type type, const uint32_t* d_rowids,
                            uint64_t n, uint64_t k, olap_order order, void* d_out_keys,
                            uint32_t* d_out_rowids, int32_t* dev_status, void* stream) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    const uint64_t kk = std::min(k, n);
    olap_status st = check_topk_args(ctx, d_keys, type, n, kk, order, d_out_keys, d_out_rowids);
    if (st != OLAP_OK) return st;
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    if (kk == 0) {
        if (dev_status) {
            cudaError_t e = cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "status reset");
        }
        return OLAP_OK;
    }
    return topk_enqueue(ctx, d_keys, type, d_rowids, n, kk, order, d_out_keys, d_out_rowids, dev_status, s,
                        nullptr);
}

}  // extern "C"

extern "C" olap_status olap_ctx_time_kernels(olap_ctx* ctx, int on) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (on && !ctx->kev[0]) {
        cudaError_t e = cudaSetDevice(ctx->device);
        for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->kev[i]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "timing events");
    }
    ctx->time_kernels = on != 0;
    return OLAP_OK;
}

extern "C" olap_status olap_ctx_launches(const olap_ctx* ctx, uint64_t* count) {
    if (!ctx || !count) return OLAP_E_INVALID;
    *count = ctx->launches;
    return OLAP_OK;
}

extern "C" olap_status olap_kernel_ms_last(olap_ctx* ctx, olap_kernel_ms* out) {
    if (!ctx || !out) return OLAP_E_INVALID;
    ctx->last_error.clear();
    out->topk_prepare_ms = out->topk_filter_ms = out->topk_select_ms = out->join_probe_ms = -1.0f;
    cudaError_t e = cudaSuccess;
    auto span = [&](int a, int b, float* ms) {
        if (e == cudaSuccess) e = cudaEventSynchronize(ctx->kev[b]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ctx->kev[a], ctx->kev[b]);
    };
    if (ctx->topk_timed) {
        span(0, 1, &out->topk_prepare_ms);
        if (ctx->topk_filtered) span(1, 2, &out->topk_filter_ms);
        span(2, 3, &out->topk_select_ms);
    }
    if (ctx->probe_timed) span(4, 5, &out->join_probe_ms);
    return e == cudaSuccess ? OLAP_OK : cuda_fail(ctx, e, "kernel timing read-back");
}

extern "C" olap_status olap_topk_info_last(olap_ctx* ctx, olap_topk_info* out) {
    if (!ctx || !out) return OLAP_E_INVALID;
    std::memset(out, 0, sizeof(*out));
    if (!ctx->last_topk_ctl) return fail(ctx, OLAP_E_INVALID, "no Top-K has run on this context");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "Top-K info");
    TopkCtl c;
    e = cudaMemcpy(&c, ctx->last_topk_ctl, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "Top-K info read-back");
    out->path = c.path;
    out->refine_passes = c.passes;
    out->candidates = c.cand_count;
    out->rowids_in_place = ctx->last_rowids_in_place ? 1 : 0;
    auto d = [&](int a, int b) { return c.ts[b] > c.ts[a] ? c.ts[b] - c.ts[a] : 0ull; };
    out->phase_ns[0] = d(0, 1);
    out->phase_ns[1] = d(1, 2);
    out->phase_ns[2] = d(2, 4);
    out->phase_ns[3] = d(4, 5);
    out->phase_ns[4] = d(5, 6);
    out->phase_ns[5] = d(0, 6);
    out->phase_ns[6] = d(5, 7);
    out->phase_ns[7] = d(7, 8);
    return OLAP_OK;
}
