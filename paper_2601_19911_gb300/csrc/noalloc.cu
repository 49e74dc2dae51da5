// Top-K for callers that cannot allocate device memory.
//
// Some callers must not have a library allocate GPU memory on their behalf:
// engines whose device memory is entirely reserved by their own pool (a
// database buffer manager, a framework's caching allocator), plug-in and UDF
// hosts that forbid allocation inside an operator, and latency-critical paths
// that cannot accept the device-wide synchronisation cudaMalloc/cudaFree may
// cause.  olap_topk_noalloc serves them: it runs the same Top-K kernels as
// olap_topk_async, but its working memory is a fixed array compiled into this
// file, so the call itself allocates nothing.  The caller still provides the
// input and output buffers.
//
// The array below lives in the memory of every GPU that has loaded this
// file's code module and stays there until the process exits.  Its address is
// looked up once per device (cudaGetSymbolAddress, with that device current)
// on the first call made on that device.  With lazy module loading (CUDA's
// default) that lookup is also what loads the module, so the first call on a
// device takes the array's 2 MiB of device memory and may synchronise; make
// it during start-up, before any stream capture.  Later calls allocate nothing.
// All calls on one device share the array and it keeps the previous call's
// contents: the grid barrier at its start is cleared before every launch, and
// the kernel clears its own counters and histograms.  Calls whose work
// overlaps on the GPU (on different streams, or from different host threads
// without ordering) race on the array and give wrong results; order them.
#include <mutex>

#include "olap.h"
#include "topk.cuh"

namespace {

// Size of the fixed working array.  It covers n <= OLAP_NOALLOC_MAX_N keys and
// k <= OLAP_NOALLOC_MAX_K at every n (the largest need, at n = 2^24 and
// k = 4096, is about 1.2 MiB with the 64 KiB sample).
constexpr size_t NOALLOC_BYTES = 2u << 20;
static_assert(OLAP_NOALLOC_MAX_N <= (1ull << 32), "row index must fit 32 bits");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;

struct DeviceSetup {
    bool done = false;
    void* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    olap::TopkGeom geom{};     // launch geometry of the Top-K kernels
};

std::mutex g_setup_lock;
DeviceSetup g_setup[MAX_DEVICES];

// Per-device set-up, done by the first call on that device (device current).
olap_status setup_device(int dev, DeviceSetup* out) {
    std::lock_guard<std::mutex> guard(g_setup_lock);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return OLAP_E_CUDA;
        }
        olap::TopkGeom g;
        if (!olap::topk_geometry(dev, 0, 0, 0, 0, &g)) {
            cudaGetLastError();
            return OLAP_E_CUDA;
        }
        s.scratch = p;
        s.geom = g;
        s.done = true;
    }
    *out = s;
    return OLAP_OK;
}

}  // namespace

extern "C" olap_status olap_topk_noalloc(const void* d_keys, olap_key_type type, const uint32_t* d_rowids,
                                         uint64_t n, uint64_t k, olap_order order, void* d_out_keys,
                                         uint32_t* d_out_rowids, int32_t* dev_status, void* stream) {
    if (type < OLAP_KEY_I64 || type > OLAP_KEY_U32) return OLAP_E_INVALID;
    if (order != OLAP_ASC && order != OLAP_DESC) return OLAP_E_INVALID;
    // Sizes beyond the fixed array are refused before anything is launched.
    if (n > OLAP_NOALLOC_MAX_N || k > OLAP_NOALLOC_MAX_K) return OLAP_E_INVALID;
    const uint64_t kk = k < n ? k : n;
    if (n && !d_keys) return OLAP_E_INVALID;
    if (kk && (!d_out_keys || !d_out_rowids)) return OLAP_E_INVALID;
    const size_t w = olap::key_bytes(type);
    if (reinterpret_cast<uintptr_t>(d_keys) % w) return OLAP_E_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kk == 0) {
        if (dev_status && cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s) != cudaSuccess) {
            cudaGetLastError();
            return OLAP_E_CUDA;
        }
        return OLAP_OK;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return OLAP_E_CUDA;
    }
    DeviceSetup ds;
    olap_status st = setup_device(dev, &ds);
    if (st != OLAP_OK) return st;

    const olap::TopkPlan plan = olap::topk_plan(n, kk);
    if (olap::topk_scratch_bytes(plan, kk) > NOALLOC_BYTES) return OLAP_E_INVALID;
    olap::TopkArgs a{};
    a.keys = d_keys;
    a.rowids = d_rowids;
    a.n = n;
    a.k = kk;
    a.kind = type;
    a.w4 = olap::key_bytes(type) == 4;
    a.desc = order == OLAP_DESC;
    olap::topk_carve(a, plan, ds.scratch);
    a.filter = olap::TK_FILTER_REGS;
    a.out_keys = d_out_keys;
    a.out_rowids = d_out_rowids;
    a.dev_status = dev_status;
    // The grid barrier must start at zero; an earlier call that gave up on a
    // wait may have left it mid-count.
    if (cudaMemsetAsync(a.bar, 0, sizeof(olap::GridBar), s) != cudaSuccess) {
        cudaGetLastError();
        return OLAP_E_CUDA;
    }
    if (olap::topk_launch(a, ds.geom, s) != cudaSuccess) {
        cudaGetLastError();
        return OLAP_E_CUDA;
    }
    return OLAP_OK;
}
