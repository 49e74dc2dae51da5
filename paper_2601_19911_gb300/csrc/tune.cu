// Autotuner: picks the radix digit width and the streaming-filter block size
// of Top-K, and the load factor, probe mode and bucket-read cache path of the
// hash join, by timing candidate configurations on device-generated tuning
// inputs of the caller's shape.  The context is left configured with the
// fastest candidates; the default configuration is timed alongside so the
// gain is reported, not assumed.
//
// Tuning inputs (not test data): Top-K keys are uniform 64-bit patterns
// (float32: their top 32 bits); build keys are distinct with high
// probability; a probe row is a hit with probability `join_hit_rate`, then it
// carries the key of a uniformly chosen build row, else a fresh random key.
// All draws are counter-based splitmix64 (Steele, Lea, Flood, OOPSLA 2014).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "topk.cuh"

namespace {

__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void gen_topk_keys(void* keys, uint64_t n, int w4, uint64_t seed) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t v = splitmix(seed, i);
        if (w4) static_cast<uint32_t*>(keys)[i] = static_cast<uint32_t>(v >> 32);
        else static_cast<uint64_t*>(keys)[i] = v;
    }
}

__global__ void gen_join_keys(int64_t* build, uint64_t nb, int64_t* probe, uint64_t np, double hit, uint64_t seed) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t t0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (uint64_t i = t0; i < nb; i += stride) build[i] = static_cast<int64_t>(splitmix(seed, i));
    for (uint64_t j = t0; j < np; j += stride) {
        const double u = static_cast<double>(splitmix(seed + 1, j) >> 11) * 0x1.0p-53;
        uint64_t v;
        if (nb && u < hit) v = splitmix(seed, splitmix(seed + 2, j) % nb);
        else v = splitmix(seed + 3, j);
        probe[j] = static_cast<int64_t>(v);
    }
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

double median(std::vector<double> v) {
    std::sort(v.begin(), v.end());
    return v.empty() ? 0.0 : v[v.size() / 2];
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

// Puts the context's options and Top-K geometry back unless the tuned values
// are committed (early returns leave the context as it was).
struct OptsGuard {
    olap_ctx* ctx;
    olap_opts opts;
    olap::TopkGeom geom;
    bool keep = false;
    explicit OptsGuard(olap_ctx* c) : ctx(c), opts(c->opts), geom(c->topk_geom) {}
    ~OptsGuard() {
        if (!keep) {
            ctx->opts = opts;
            ctx->topk_geom = geom;
        }
    }
};

}  // namespace

using namespace olap;

extern "C" olap_status olap_autotune(olap_ctx* ctx, const olap_tune_request* req, olap_tune_result* out) {
    if (!ctx) return OLAP_E_INVALID;
    ctx->last_error.clear();
    if (!req || !out) return fail(ctx, OLAP_E_INVALID, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    if (req->topk_n >= (1ull << 32) || req->join_probe_n >= (1ull << 32) || req->join_build_n >= (1ull << 32))
        return fail(ctx, OLAP_E_INVALID, "tuning sizes must be below 2^32");
    if (req->topk_n && (req->topk_key_type < OLAP_KEY_I64 || req->topk_key_type > OLAP_KEY_U32))
        return fail(ctx, OLAP_E_INVALID, "bad key type");
    if (req->join_probe_n && !req->join_build_n) return fail(ctx, OLAP_E_INVALID, "probe without build rows");
    if (!(req->join_hit_rate >= 0.0 && req->join_hit_rate <= 1.0)) return fail(ctx, OLAP_E_INVALID, "bad hit rate");
    const int reps = req->reps > 0 ? req->reps : 5;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set device");
    Events ev;
    if ((e = cudaEventCreate(&ev.a)) != cudaSuccess || (e = cudaEventCreate(&ev.b)) != cudaSuccess)
        return cuda_fail(ctx, e, "tuning events");
    cudaStream_t s = ctx->stream;
    int tried = 0;
    // Median device time of `reps` runs of fn (after one untimed run).
    auto timed = [&](auto fn, double* ms) -> olap_status {
        olap_status st = fn();
        if (st != OLAP_OK) return st;
        std::vector<double> t;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(ev.a, s);
            if ((st = fn()) != OLAP_OK) return st;
            cudaEventRecord(ev.b, s);
            if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess) return cuda_fail(ctx, e, "tuning run");
            float f = 0.f;
            cudaEventElapsedTime(&f, ev.a, ev.b);
            t.push_back(f);
        }
        *ms = median(t);
        ++tried;
        return OLAP_OK;
    };

    // ---- Top-K: filter block size, then digit width --------------------------
    if (req->topk_n) {
        const uint64_t n = req->topk_n, kk = std::min<uint64_t>(std::max<uint64_t>(req->topk_k, 1), n);
        const bool w4 = key_bytes(req->topk_key_type) == 4;
        const size_t w = w4 ? 4 : 8;
        DevBuf keys, ok, orow;
        if ((e = cudaMalloc(&keys.p, n * w)) != cudaSuccess || (e = cudaMalloc(&ok.p, kk * w)) != cudaSuccess ||
            (e = cudaMalloc(&orow.p, kk * 4)) != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(ctx, e, "tuning allocation");
        }
        gen_topk_keys<<<ctx->sm_count * 4, 256, 0, s>>>(keys.p, n, w4 ? 1 : 0, req->seed);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "tuning input");
        ctx->launches += 1;
        const olap_key_type kt = static_cast<olap_key_type>(req->topk_key_type);
        auto run = [&]() {
            return olap_topk_async(ctx, keys.p, kt, nullptr, n, kk, OLAP_DESC, ok.p, static_cast<uint32_t*>(orow.p),
                                   nullptr, nullptr);
        };
        OptsGuard guard(ctx);
        auto configure = [&](int block, int digit) -> bool {
            TopkGeom g;
            if (!topk_geometry(ctx->device, ctx->opts.topk_tile_bytes, ctx->opts.topk_stages,
                               ctx->opts.topk_ctas_per_sm, block, &g))
                return false;
            ctx->topk_geom = g;
            ctx->opts.block_threads = block;
            ctx->opts.topk_digit_bits = digit;
            return true;
        };
        double best = 0.0, t = 0.0;
        int best_block = 512, best_digit = 12;
        olap_status st;
        if (!configure(512, 12)) return fail(ctx, OLAP_E_CUDA, "default Top-K geometry");
        if ((st = timed(run, &t)) != OLAP_OK) return st;
        out->topk_default_ms = t;
        best = t;
        for (int block : {256, 1024}) {
            if (!configure(block, 12)) continue;
            if ((st = timed(run, &t)) != OLAP_OK) return st;
            if (t < best) best = t, best_block = block;
        }
        for (int digit : {8, 10, 11}) {
            if (!configure(best_block, digit)) continue;
            if ((st = timed(run, &t)) != OLAP_OK) return st;
            if (t < best) best = t, best_digit = digit;
        }
        if (!configure(best_block, best_digit)) return fail(ctx, OLAP_E_CUDA, "tuned Top-K geometry");
        guard.keep = true;
        out->block_threads = best_block;
        out->topk_digit_bits = best_digit;
        out->topk_ms = best;
    }

    // ---- Join: load factor, probe mode, bucket-read path ----------------------
    if (req->join_build_n) {
        const uint64_t nb = req->join_build_n, np = req->join_probe_n;
        const uint64_t cap = std::max<uint64_t>(1, static_cast<uint64_t>(
                                                       std::ceil(static_cast<double>(np) * 1.05 + 4096.0)));
        DevBuf bk, pk, pairs, cnt;
        if ((e = cudaMalloc(&bk.p, nb * 8)) != cudaSuccess || (e = cudaMalloc(&pk.p, std::max<uint64_t>(np, 1) * 8)) !=
            cudaSuccess || (e = cudaMalloc(&pairs.p, cap * 8)) != cudaSuccess ||
            (e = cudaMalloc(&cnt.p, 256)) != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(ctx, e, "tuning allocation");
        }
        gen_join_keys<<<ctx->sm_count * 4, 256, 0, s>>>(static_cast<int64_t*>(bk.p), nb, static_cast<int64_t*>(pk.p),
                                                       np, req->join_hit_rate, req->seed + 16);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "tuning input");
        ctx->launches += 1;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "tuning input");
        const olap_opts saved = ctx->opts;
        double best = -1.0, t = 0.0;
        double best_load = 0.5, best_build = 0.0;
        int best_parts = 0, best_loads = OLAP_LOADS_L2_ONLY;
        olap_status st;
        for (double load : {0.25, 0.35, 0.5, 0.7}) {
            olap_join_table* table = nullptr;
            double build_ms = 0.0;
            auto build = [&]() {
                if (table) olap_join_free(table);
                table = nullptr;
                return olap_join_build(ctx, static_cast<const int64_t*>(bk.p), nullptr, OLAP_MEM_DEVICE, nb, load,
                                       &table);
            };
            if ((st = timed(build, &build_ms)) != OLAP_OK) {
                if (table) olap_join_free(table);
                if (st == OLAP_E_NOMEM) continue;    // this load factor does not fit the budget
                ctx->opts = saved;
                return st;
            }
            for (int parts : {0, 1}) {
                for (int loads : {OLAP_LOADS_L1, OLAP_LOADS_L2_ONLY}) {
                    ctx->opts.join_partitions = parts;
                    ctx->opts.join_bucket_loads = loads;
                    auto probe = [&]() {
                        return olap_join_probe_async(ctx, table, static_cast<const int64_t*>(pk.p), nullptr, np,
                                                     static_cast<olap_pair*>(pairs.p), cap,
                                                     static_cast<uint64_t*>(cnt.p), nullptr);
                    };
                    if ((st = timed(probe, &t)) != OLAP_OK) {
                        olap_join_free(table);
                        ctx->opts = saved;
                        return st;
                    }
                    if (load == 0.5 && parts == 0 && loads == OLAP_LOADS_L2_ONLY) out->join_probe_default_ms = t;
                    if (best < 0.0 || t < best) {
                        best = t;
                        best_load = load;
                        best_parts = parts;
                        best_loads = loads;
                        best_build = build_ms;
                    }
                }
            }
            olap_join_free(table);
        }
        ctx->opts = saved;
        if (best < 0.0) return fail(ctx, OLAP_E_NOMEM, "no join candidate fits the memory budget");
        ctx->opts.load_factor = best_load;
        ctx->opts.join_partitions = best_parts;
        ctx->opts.join_bucket_loads = best_loads;
        out->load_factor = best_load;
        out->join_partitions = best_parts;
        out->join_bucket_loads = best_loads;
        out->join_probe_ms = best;
        out->join_build_ms = best_build;
    }
    out->candidates = tried;
    return OLAP_OK;
}
