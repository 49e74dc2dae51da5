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
// Probe: every thread takes JP_U probe keys per round (coalesced loads),
// issues their first bucket loads together, then walks the chains in
// warp-uniform steps.  Matches are appended per warp (one ballot per slot)
// into a per-CTA shared-memory stage that is flushed to the output in blocks
// of at least JP_FLUSH pairs with one atomic on the global count.
#include <algorithm>
#include <cstring>
#include <string>

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

__global__ void __launch_bounds__(JP_TPB, 4) join_probe_kernel(ProbeArgs a) {
    extern __shared__ __align__(16) uint2 stage[];
    __shared__ unsigned scount;
    __shared__ unsigned long long sbase;
    probe_rounds(a, blockIdx.x, gridDim.x, a.n, stage, &scount, &sbase);
}

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

int probe_grid(int device) {
    static int cached[64] = {};
    if (device < 0 || device >= 64) return 0;
    if (cached[device]) return cached[device];
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(join_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, JP_SMEM) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, join_probe_kernel, JP_TPB, JP_SMEM) != cudaSuccess)
        return 0;
    cached[device] = sms * std::max(1, per);
    return cached[device];
}

}  // namespace

}  // namespace olap


using namespace olap;

namespace {

olap_status probe_enqueue(olap_ctx* ctx, const olap_join_table* t, const int64_t* d_keys, const uint32_t* d_rowids,
                          uint64_t n, olap_pair* d_out, uint64_t capacity, uint64_t* d_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "probe count reset");
    if (n == 0) return OLAP_OK;
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
    ctx->probe_timed = ctx->time_kernels;
    if (ctx->time_kernels && (e = cudaEventRecord(ctx->kev[4], s)) != cudaSuccess)
        return cuda_fail(ctx, e, "timing event");
    join_probe_kernel<<<grid, JP_TPB, JP_SMEM, s>>>(a);
    e = cudaGetLastError();
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
    const size_t slot_bytes = buckets * 32;
    const size_t bytes = slot_bytes + 256;
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
    e = cudaMemsetAsync(mem, 0xFF, slot_bytes, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(jc, 0, sizeof(JoinCtl), ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "join table init"));
    if (n) {
        const int grid = ctx->sm_count * 8;
        join_build_kernel<<<grid, JB_TPB, 0, ctx->stream>>>(dk, dr, n, t->slots, buckets - 1, jc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "build launch"));
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

olap_status olap_join_table_info(const olap_join_table* t, uint64_t* n_build, uint64_t* n_buckets, uint64_t* n_side) {
    if (!t || !t->slots) return OLAP_E_INVALID;
    if (n_build) *n_build = t->n_build;
    if (n_buckets) *n_buckets = t->n_buckets;
    if (n_side) *n_side = t->n_side;
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
