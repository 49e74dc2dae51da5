// Host engine used by the serving harness for the requests the gate keeps on
// the CPU: the "existing execution engine" of the paper's hybrid design
// (Sec. II-A) that the GPU augments.  It is a separate library on purpose:
// the GPU library has no CPU implementation of the primitives.
//
//   Top-K: each thread keeps the K smallest composites (order-preserving key
//   word, row-id) of its chunk -- a bounded max-heap when K is small against
//   the chunk, else nth_element over the chunk -- then the K smallest of the
//   union are selected with nth_element and sorted.  Same ordering as the
//   GPU: key in the requested order, row-id ascending on ties, float32 by IEEE
//   totalOrder.
//   Probe: per table, rows sorted by key plus an open-addressing index from
//   key to its run; threads probe chunks and the pairs are concatenated.
#include <pthread.h>
#include <sched.h>

#include <algorithm>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <queue>
#include <thread>
#include <vector>

#include "olap.h"

namespace {

struct Comp {
    uint64_t r;
    uint32_t rid;
    bool operator<(const Comp& o) const { return r < o.r || (r == o.r && rid < o.rid); }
};

// Order-preserving word of a key (4-byte keys in the low half of `bits`):
// signed integers offset by the sign bit, unsigned as they are, floats by
// IEEE 754 totalOrder (negatives inverted, non-negatives with the sign bit
// set); complemented for DESC.  And its inverse.
inline bool wide(int kind) { return kind == OLAP_KEY_I64 || kind == OLAP_KEY_F64 || kind == OLAP_KEY_U64; }

inline uint64_t word(uint64_t bits, int kind, bool desc) {
    uint64_t u;
    switch (kind) {
        case OLAP_KEY_I64: u = bits ^ 0x8000000000000000ull; break;
        case OLAP_KEY_U64: u = bits; break;
        case OLAP_KEY_F64: u = (bits >> 63) ? ~bits : (bits | 0x8000000000000000ull); break;
        case OLAP_KEY_I32: u = static_cast<uint32_t>(bits) ^ 0x80000000u; break;
        case OLAP_KEY_U32: u = static_cast<uint32_t>(bits); break;
        default: {
            const uint32_t b = static_cast<uint32_t>(bits);
            u = (b >> 31) ? static_cast<uint32_t>(~b) : (b | 0x80000000u);
        }
    }
    if (desc) u = wide(kind) ? ~u : (~u & 0xFFFFFFFFull);
    return u;
}

inline uint64_t unword(uint64_t r, int kind, bool desc) {
    uint64_t u = desc ? (wide(kind) ? ~r : (~r & 0xFFFFFFFFull)) : r;
    switch (kind) {
        case OLAP_KEY_I64: return u ^ 0x8000000000000000ull;
        case OLAP_KEY_U64: return u;
        case OLAP_KEY_F64: return (u >> 63) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
        case OLAP_KEY_I32: return static_cast<uint32_t>(u) ^ 0x80000000u;
        case OLAP_KEY_U32: return static_cast<uint32_t>(u);
        default: {
            const uint32_t v = static_cast<uint32_t>(u);
            return (v >> 31) ? (v & 0x7FFFFFFFu) : static_cast<uint32_t>(~v);
        }
    }
}

struct Table {
    std::vector<int64_t> keys;      // sorted
    std::vector<uint32_t> rids;     // in key order
    std::vector<uint64_t> slot_key; // index: key -> first position, count
    std::vector<uint32_t> slot_pos, slot_cnt;
    uint64_t mask = 0;
};

inline uint64_t mix(uint64_t h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

// Persistent worker threads: a request's chunks are queued to them, so a
// parallel request costs a queue hand-off rather than thread creation.
// Tasks never wait on other tasks, so concurrent requests cannot deadlock.
// Pins the calling thread (or `th`) to the given host cores; an empty set
// leaves it where it is.  Returns false if the system refuses.
bool pin_to(pthread_t th, const std::vector<int>& cpus) {
    if (cpus.empty()) return true;
    cpu_set_t set;
    CPU_ZERO(&set);
    for (int c : cpus)
        if (c >= 0 && c < CPU_SETSIZE) CPU_SET(c, &set);
    return pthread_setaffinity_np(th, sizeof(set), &set) == 0;
}

class Pool {
public:
    Pool(int n, const std::vector<int>& cpus) {
        for (int i = 0; i < n; ++i) {
            th_.emplace_back([this] { loop(); });
            pin_to(th_.back().native_handle(), cpus);
        }
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
    }
    void post(std::function<void()> f) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            q_.push_back(std::move(f));
        }
        cv_.notify_one();
    }

private:
    void loop() {
        while (true) {
            std::function<void()> f;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
                if (q_.empty()) return;
                f = std::move(q_.front());
                q_.pop_front();
            }
            f();
        }
    }
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<std::function<void()>> q_;
    std::vector<std::thread> th_;
    bool stop_ = false;
};

struct Engine {
    int threads = 8;
    std::vector<int> cpus;             // host cores the engine computes on (empty: anywhere)
    std::vector<Table> tables;
    Pool* pool = nullptr;
    ~Engine() { delete pool; }
};

// A request computes its first chunk on the calling thread (a serving loop's
// host worker), so with a core set the caller is pinned to it as well, once.
void pin_caller(const Engine* E) {
    thread_local const Engine* pinned_for = nullptr;
    if (E->cpus.empty() || pinned_for == E) return;
    pin_to(pthread_self(), E->cpus);
    pinned_for = E;
}

constexpr uint64_t TOPK_CHUNK = 65536;    // rows per thread at least: Top-K (streaming)
constexpr uint64_t PROBE_CHUNK = 8192;    // probe (a random table access per row)

// Chunks a request of n rows is cut into.
int chunks_for(const Engine* E, uint64_t n, uint64_t min_chunk) {
    return static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(E->threads, n / min_chunk)));
}

// Run f(i, a, b) over t chunks of [0, n): chunk 0 on the calling thread, the
// others on the pool; returns when all are done.
template <typename F>
void parallel(Engine* E, int t, uint64_t n, F&& f) {
    if (t <= 1) {
        f(0, 0, n);
        return;
    }
    const uint64_t per = (n + t - 1) / t;
    std::mutex mu;
    std::condition_variable cv;
    int left = t - 1;
    for (int i = 1; i < t; ++i) {
        const uint64_t a = std::min(n, i * per), b = std::min(n, a + per);
        E->pool->post([&, i, a, b] {
            f(i, a, b);
            std::lock_guard<std::mutex> lk(mu);
            if (--left == 0) cv.notify_one();
        });
    }
    f(0, 0, std::min(n, per));
    std::unique_lock<std::mutex> lk(mu);
    cv.wait(lk, [&] { return left == 0; });
}

int run_topk(Engine* E, olap_serve_request* r) {
    const int kind = r->key_type;
    const bool desc = r->order == OLAP_DESC, w8 = wide(kind);
    const uint64_t n = r->n, kk = std::min(r->k, n);
    if (kk == 0) {
        r->out_count = 0;
        return OLAP_OK;
    }
    const int t = chunks_for(E, n, TOPK_CHUNK);
    std::vector<std::vector<Comp>> part(t);
    auto comp = [&](uint64_t i) {
        Comp c;
        c.r = word(w8 ? static_cast<const uint64_t*>(r->keys)[i] : static_cast<const uint32_t*>(r->keys)[i], kind,
                   desc);
        c.rid = r->rowids ? r->rowids[i] : static_cast<uint32_t>(i);
        return c;
    };
    parallel(E, t, n, [&](int ti, uint64_t a, uint64_t b) {
        auto& v = part[ti];
        if (kk * 16 >= b - a) {                 // K large against the chunk: select
            v.resize(b - a);
            for (uint64_t i = a; i < b; ++i) v[i - a] = comp(i);
            if (v.size() > kk) {
                std::nth_element(v.begin(), v.begin() + static_cast<long>(kk), v.end());
                v.resize(kk);
            }
            return;
        }
        std::priority_queue<Comp> heap;
        for (uint64_t i = a; i < b; ++i) {
            const Comp c = comp(i);
            if (heap.size() < kk) heap.push(c);
            else if (c < heap.top()) {
                heap.pop();
                heap.push(c);
            }
        }
        v.reserve(heap.size());
        while (!heap.empty()) {
            v.push_back(heap.top());
            heap.pop();
        }
    });
    std::vector<Comp> all;
    for (auto& v : part) all.insert(all.end(), v.begin(), v.end());
    if (all.size() > kk) std::nth_element(all.begin(), all.begin() + static_cast<long>(kk), all.end());
    std::sort(all.begin(), all.begin() + static_cast<long>(kk));
    for (uint64_t i = 0; i < kk; ++i) {
        if (w8) static_cast<uint64_t*>(r->out_keys)[i] = unword(all[i].r, kind, desc);
        else static_cast<uint32_t*>(r->out_keys)[i] = static_cast<uint32_t>(unword(all[i].r, kind, desc));
        r->out_rowids[i] = all[i].rid;
    }
    r->out_count = kk;
    return OLAP_OK;
}

int run_probe(Engine* E, olap_serve_request* r) {
    if (r->table_id < 0 || r->table_id >= static_cast<int>(E->tables.size())) return OLAP_E_INVALID;
    const Table& T = E->tables[r->table_id];
    const int64_t* keys = static_cast<const int64_t*>(r->keys);
    const int t = chunks_for(E, r->n, PROBE_CHUNK);
    std::vector<std::vector<olap_pair>> part(t);
    parallel(E, t, r->n, [&](int ti, uint64_t a, uint64_t b) {
        auto& v = part[ti];
        for (uint64_t i = a; i < b; ++i) {
            const uint64_t key = static_cast<uint64_t>(keys[i]);
            uint64_t s = mix(key) & T.mask;
            while (T.slot_cnt[s]) {
                if (T.slot_key[s] == key) {
                    const uint32_t prid = r->rowids ? r->rowids[i] : static_cast<uint32_t>(i);
                    for (uint32_t j = 0; j < T.slot_cnt[s]; ++j) v.push_back(olap_pair{prid, T.rids[T.slot_pos[s] + j]});
                    break;
                }
                s = (s + 1) & T.mask;
            }
        }
    });
    uint64_t total = 0;
    for (auto& v : part) total += v.size();
    r->out_count = total;
    if (total > r->capacity) return OLAP_E_OVERFLOW;
    uint64_t off = 0;
    for (auto& v : part) {
        if (!v.empty()) std::memcpy(r->out_pairs + off, v.data(), v.size() * sizeof(olap_pair));
        off += v.size();
    }
    return OLAP_OK;
}

}  // namespace

extern "C" {

void* olap_host_engine_create(int threads) {
    Engine* e = new Engine();
    e->threads = threads > 0 ? threads : 8;
    e->pool = new Pool(e->threads, e->cpus);
    return e;
}

// The same, computing only on the given host cores (its pool threads, and
// every thread that calls olap_host_engine_run), so that it leaves the other
// cores to whatever else runs in the process (a GPU path's staging copies).
void* olap_host_engine_create_on(int threads, const int* cpus, int ncpus) {
    Engine* e = new Engine();
    e->threads = threads > 0 ? threads : 8;
    if (cpus)
        for (int i = 0; i < ncpus; ++i) e->cpus.push_back(cpus[i]);
    e->pool = new Pool(e->threads, e->cpus);
    return e;
}

int olap_host_engine_add_table(void* eng, const int64_t* keys, const uint32_t* rowids, uint64_t n) {
    Engine* E = static_cast<Engine*>(eng);
    Table T;
    std::vector<uint64_t> idx(n);
    for (uint64_t i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t b) { return keys[a] < keys[b]; });
    T.keys.resize(n);
    T.rids.resize(n);
    for (uint64_t i = 0; i < n; ++i) {
        T.keys[i] = keys[idx[i]];
        T.rids[i] = rowids ? rowids[idx[i]] : static_cast<uint32_t>(idx[i]);
    }
    uint64_t cap = 1;
    while (cap < 2 * n + 2) cap <<= 1;
    T.mask = cap - 1;
    T.slot_key.assign(cap, 0);
    T.slot_pos.assign(cap, 0);
    T.slot_cnt.assign(cap, 0);
    for (uint64_t i = 0; i < n;) {
        uint64_t j = i;
        while (j < n && T.keys[j] == T.keys[i]) ++j;
        const uint64_t key = static_cast<uint64_t>(T.keys[i]);
        uint64_t s = mix(key) & T.mask;
        while (T.slot_cnt[s]) s = (s + 1) & T.mask;
        T.slot_key[s] = key;
        T.slot_pos[s] = static_cast<uint32_t>(i);
        T.slot_cnt[s] = static_cast<uint32_t>(j - i);
        i = j;
    }
    E->tables.push_back(std::move(T));
    return static_cast<int>(E->tables.size()) - 1;
}

int olap_host_engine_run(void* eng, olap_serve_request* r) {
    Engine* E = static_cast<Engine*>(eng);
    pin_caller(E);
    if (r->op == OLAP_OP_TOPK) return run_topk(E, r);
    if (r->op == OLAP_OP_PROBE) return run_probe(E, r);
    return OLAP_E_INVALID;
}

// Cut the key column out of a row table (a row store's key-only extraction,
// Sec. V-C): key i = the key_width bytes at rows + i * row_bytes + key_offset.
void olap_host_engine_extract(void* eng, const void* rows, uint64_t n, uint32_t row_bytes, uint32_t key_offset,
                              uint32_t key_width, void* out) {
    Engine* E = static_cast<Engine*>(eng);
    const unsigned char* r = static_cast<const unsigned char*>(rows);
    unsigned char* o = static_cast<unsigned char*>(out);
    parallel(E, chunks_for(E, n, TOPK_CHUNK), n, [&](int, uint64_t a, uint64_t b) {
        if (key_width == 8)
            for (uint64_t i = a; i < b; ++i) std::memcpy(o + i * 8, r + i * row_bytes + key_offset, 8);
        else
            for (uint64_t i = a; i < b; ++i) std::memcpy(o + i * key_width, r + i * row_bytes + key_offset, key_width);
    });
}

// Smallest request size the engine runs on more than one thread (0 if it
// never does): where its cost changes regime, for the gate's CPU model.
uint64_t olap_host_engine_parallel_from(void* eng, int op) {
    const Engine* E = static_cast<const Engine*>(eng);
    if (E->threads < 2) return 0;
    return 2 * (op == OLAP_OP_TOPK ? TOPK_CHUNK : PROBE_CHUNK);
}

void olap_host_engine_free(void* eng) { delete static_cast<Engine*>(eng); }

}  // extern "C"
