// Serving loop with continuous batching and the Risky Gate (Sec. II-B: offload
// only when the estimated gain exceeds the margin; Sec. IV: gated against
// always-on offload, tail latency).
//
// One dispatcher thread releases requests at their arrival times and decides
// where each runs.  GPU requests wait in one FIFO; gpu_slots slot threads,
// each with its own context (stream, scratch, pinned double buffers), take the
// head of the FIFO as soon as its device memory fits the budget next to the
// requests in flight, so work of different requests overlaps on the device.
// Host requests go to cpu_workers threads that call the caller's engine.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "ctx.h"
#include "topk.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// Device bytes one GPU request holds while it runs: its key-only input, the
// selection scratch or the pair output (and probe partitions), and its result
// staging.  `ctx` (any slot context, all alike) decides the probe mode.
uint64_t device_need(const olap_serve_request& r, const olap_ctx* ctx) {
    const uint64_t rid = r.rowids ? 4 * r.n : 0;
    if (r.op == OLAP_OP_TOPK) {
        const uint64_t w = olap::key_bytes(r.key_type);
        const uint64_t kk = std::min(r.k, r.n);
        return r.n * w + rid + olap::topk_scratch_bytes(olap::topk_plan(r.n, kk), kk) + kk * (w + 4) + 4096;
    }
    const uint64_t part = ctx && r.table ? olap::probe_scratch_bytes(ctx, r.table, r.n) : 0;
    return r.n * 8 + rid + r.capacity * 8 + part + 4096;
}

bool decide_gpu(const olap_serve_request& r, const olap_serve_opts& o) {
    if (o.policy == OLAP_SERVE_ALWAYS_GPU) return true;
    if (o.policy == OLAP_SERVE_ALWAYS_HOST) return false;
    olap_gate_query q;
    std::memset(&q, 0, sizeof(q));
    q.n = r.n;
    const double nd = static_cast<double>(r.n);
    const double rid = r.rowids ? 4.0 : 0.0;
    olap_gate_decision d;
    if (r.op == OLAP_OP_TOPK) {
        const double w = olap::key_bytes(r.key_type);
        q.op = OLAP_OP_TOPK;
        q.k_or_m = static_cast<double>(r.k);
        q.tx_bytes = nd * (w + rid);
        q.out_rows = std::min(static_cast<double>(r.k), nd);
        q.bytes_per_row = w + rid;
        if (olap_gate_estimate(o.topk_model, &q, &d) != OLAP_OK) return true;
    } else {
        q.op = OLAP_OP_PROBE;
        q.k_or_m = nd > 0 ? 1.0 + r.expected_pairs / nd : 1.0;
        q.tx_bytes = nd * (8.0 + rid);
        q.out_rows = r.expected_pairs;
        q.bytes_per_row = 8.0 + rid;
        q.out_per_row = nd > 0 ? r.expected_pairs / nd : 0.0;
        if (olap_gate_estimate(o.probe_model, &q, &d) != OLAP_OK) return true;
    }
    return d.offload != 0;
}

struct Server {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> gpu_q, host_q;
    bool arrivals_done = false;
    uint64_t reserved = 0, peak = 0, budget = 0;
    olap_serve_request* reqs = nullptr;
    std::vector<uint64_t> need;
    Clock::time_point t0;
};

void gpu_slot(Server* S, olap_ctx* ctx) {
    while (true) {
        uint64_t i;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] {
                if (S->gpu_q.empty()) return S->arrivals_done;
                const uint64_t h = S->gpu_q.front();
                return S->budget == 0 || S->reserved == 0 || S->reserved + S->need[h] <= S->budget;
            });
            if (S->gpu_q.empty()) return;
            i = S->gpu_q.front();
            S->gpu_q.pop_front();
            S->reserved += S->need[i];
            S->peak = std::max(S->peak, S->reserved);
        }
        olap_serve_request& r = S->reqs[i];
        r.start_ms = ms_since(S->t0);
        uint64_t cnt = 0;
        olap_status st;
        if (r.op == OLAP_OP_TOPK) {
            st = olap_topk(ctx, r.keys, static_cast<olap_key_type>(r.key_type), r.rowids, OLAP_MEM_HOST, r.n, r.k,
                           static_cast<olap_order>(r.order), r.out_keys, r.out_rowids, OLAP_MEM_HOST, &cnt);
        } else {
            st = olap_join_probe(ctx, r.table, static_cast<const int64_t*>(r.keys), r.rowids, OLAP_MEM_HOST, r.n,
                                 r.out_pairs, OLAP_MEM_HOST, r.capacity, &cnt);
        }
        r.done_ms = ms_since(S->t0);
        r.out_count = cnt;
        r.status = st;
        r.on_gpu = 1;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->reserved -= S->need[i];
        }
        S->cv.notify_all();
    }
}

void host_worker(Server* S, const olap_serve_opts* o) {
    while (true) {
        uint64_t i;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return !S->host_q.empty() || S->arrivals_done; });
            if (S->host_q.empty()) return;
            i = S->host_q.front();
            S->host_q.pop_front();
        }
        olap_serve_request& r = S->reqs[i];
        r.start_ms = ms_since(S->t0);
        r.status = o->host_engine ? o->host_engine(o->host_user, &r) : OLAP_E_INVALID;
        r.done_ms = ms_since(S->t0);
        r.on_gpu = 0;
    }
}

double percentile(const std::vector<double>& sorted, double p) {
    if (sorted.empty()) return 0.0;
    size_t idx = static_cast<size_t>(std::ceil(p / 100.0 * static_cast<double>(sorted.size())));
    idx = idx == 0 ? 0 : idx - 1;
    return sorted[std::min(idx, sorted.size() - 1)];
}

}  // namespace

extern "C" olap_status olap_serve(olap_serve_request* reqs, uint64_t n, const olap_serve_opts* opts,
                                  olap_serve_stats* out) {
    if (!opts || !out || (n && !reqs)) return OLAP_E_INVALID;
    const olap_serve_opts o = *opts;
    if (o.policy < OLAP_SERVE_GATED || o.policy > OLAP_SERVE_ALWAYS_HOST) return OLAP_E_INVALID;
    if (o.policy == OLAP_SERVE_GATED && (!o.topk_model || !o.probe_model)) return OLAP_E_INVALID;
    if (o.policy != OLAP_SERVE_ALWAYS_GPU && !o.host_engine) return OLAP_E_INVALID;
    const int slots = o.gpu_slots > 0 ? o.gpu_slots : 4;
    const int workers = o.cpu_workers > 0 ? o.cpu_workers : 8;

    Server S;
    S.reqs = reqs;
    S.budget = o.mem_budget_bytes;
    S.need.resize(n);
    std::vector<uint64_t> order(n);
    std::iota(order.begin(), order.end(), 0ull);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint64_t a, uint64_t b) { return reqs[a].arrival_ms < reqs[b].arrival_ms; });
    std::vector<olap_ctx*> ctxs;
    auto cleanup = [&]() {
        for (olap_ctx* c : ctxs) olap_ctx_destroy(c);
    };
    if (o.policy != OLAP_SERVE_ALWAYS_HOST) {
        for (int s = 0; s < slots; ++s) {
            olap_ctx* c = nullptr;
            olap_status st = olap_ctx_create(o.ctx_opts, &c);
            if (st != OLAP_OK) {
                cleanup();
                return st;
            }
            ctxs.push_back(c);
        }
    }
    // Per-request device need, and the largest buffers a slot can be asked for,
    // so no slot allocates (and synchronises the device) while serving.
    uint64_t max_in = 0, max_out = 0, max_scratch = 0, max_part = 0;
    for (uint64_t i = 0; i < n; ++i) {
        olap_serve_request& r = reqs[i];
        r.status = OLAP_E_INVALID;
        r.out_count = 0;
        r.on_gpu = 0;
        r.start_ms = r.done_ms = 0.0;
        S.need[i] = device_need(r, ctxs.empty() ? nullptr : ctxs[0]);
        const uint64_t rid = r.rowids ? 4 * r.n : 0;
        if (r.op == OLAP_OP_TOPK) {
            const uint64_t w = olap::key_bytes(r.key_type);
            const uint64_t kk = std::min(r.k, r.n);
            max_in = std::max<uint64_t>(max_in, ((r.n * w + 255) & ~255ull) + rid);
            max_out = std::max<uint64_t>(max_out, ((kk * w + 255) & ~255ull) + kk * 4);
            max_scratch = std::max<uint64_t>(max_scratch, olap::topk_scratch_bytes(olap::topk_plan(r.n, kk), kk));
        } else {
            max_in = std::max<uint64_t>(max_in, ((r.n * 8 + 255) & ~255ull) + rid);
            max_out = std::max<uint64_t>(max_out, ((r.capacity * 8 + 255) & ~255ull) + 256);
            if (!ctxs.empty() && r.table)
                max_part = std::max<uint64_t>(max_part, olap::probe_scratch_bytes(ctxs[0], r.table, r.n));
        }
    }
    for (olap_ctx* c : ctxs) {
        olap_status st;
        if ((st = olap::ensure_dev_in(c, max_in)) != OLAP_OK || (st = olap::ensure_dev_out(c, max_out)) != OLAP_OK ||
            (st = olap::ensure_scratch(c, std::max<uint64_t>(max_scratch, 4096))) != OLAP_OK ||
            (max_part && (st = olap::ensure_part(c, max_part)) != OLAP_OK) || (st = olap::ensure_pinned(c)) != OLAP_OK) {
            cleanup();
            return st;
        }
        cudaStreamSynchronize(c->stream);
    }
    std::vector<std::thread> threads;
    S.t0 = Clock::now();
    for (olap_ctx* c : ctxs) threads.emplace_back(gpu_slot, &S, c);
    if (o.policy != OLAP_SERVE_ALWAYS_GPU)
        for (int w = 0; w < workers; ++w) threads.emplace_back(host_worker, &S, &o);
    uint64_t n_gpu = 0, n_host = 0;
    for (uint64_t j = 0; j < n; ++j) {
        const uint64_t i = order[j];
        if (!o.closed_loop) {
            const auto due = S.t0 + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double, std::milli>(reqs[i].arrival_ms));
            std::this_thread::sleep_until(due);
        }
        const bool gpu = decide_gpu(reqs[i], o);
        {
            std::lock_guard<std::mutex> lk(S.mu);
            if (gpu) {
                S.gpu_q.push_back(i);
                ++n_gpu;
            } else {
                S.host_q.push_back(i);
                ++n_host;
            }
        }
        S.cv.notify_all();
    }
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.arrivals_done = true;
    }
    S.cv.notify_all();
    for (std::thread& t : threads) t.join();
    cleanup();

    std::vector<double> lat;
    lat.reserve(n);
    double wall = 0.0, sum = 0.0;
    uint64_t failed = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const olap_serve_request& r = reqs[i];
        const double l = r.done_ms - (o.closed_loop ? 0.0 : r.arrival_ms);
        lat.push_back(l);
        sum += l;
        wall = std::max(wall, r.done_ms);
        if (r.status != OLAP_OK) ++failed;
    }
    std::sort(lat.begin(), lat.end());
    std::memset(out, 0, sizeof(*out));
    out->wall_ms = wall;
    out->throughput_rps = wall > 0 ? static_cast<double>(n) / (wall / 1e3) : 0.0;
    out->p50_ms = percentile(lat, 50);
    out->p95_ms = percentile(lat, 95);
    out->p99_ms = percentile(lat, 99);
    out->mean_ms = n ? sum / static_cast<double>(n) : 0.0;
    out->max_ms = lat.empty() ? 0.0 : lat.back();
    out->n_gpu = n_gpu;
    out->n_host = n_host;
    out->n_failed = failed;
    out->offload_fraction = n ? static_cast<double>(n_gpu) / static_cast<double>(n) : 0.0;
    out->peak_reserved_bytes = S.peak;
    return OLAP_OK;
}
