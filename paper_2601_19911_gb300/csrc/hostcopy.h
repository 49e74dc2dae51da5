// A small pool of host threads that splits one large memcpy between pageable
// and pinned host memory, so staging through the pinned buffers is not held
// to one core's copy rate.
#pragma once

#include <condition_variable>
#include <cstddef>
#include <mutex>
#include <thread>
#include <vector>

namespace olap {

class HostCopyPool {
public:
    // `helpers` threads besides the caller (0: the caller copies alone).
    explicit HostCopyPool(int helpers);
    ~HostCopyPool();
    HostCopyPool(const HostCopyPool&) = delete;
    HostCopyPool& operator=(const HostCopyPool&) = delete;

    // Copy `bytes` from src to dst with the caller and the helpers; returns
    // when every piece is done.  One copy at a time per pool.
    void copy(void* dst, const void* src, size_t bytes);

private:
    void work(int id);
    void run_pieces();

    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable go_, done_;
    unsigned long long gen_ = 0;     // job generation, bumped per copy
    bool stop_ = false;
    unsigned char* dst_ = nullptr;
    const unsigned char* src_ = nullptr;
    size_t bytes_ = 0, piece_ = 0, pieces_ = 0;
    size_t next_ = 0;                // next piece to take (under mu_)
    size_t finished_ = 0;            // pieces done (under mu_)
};

}  // namespace olap
