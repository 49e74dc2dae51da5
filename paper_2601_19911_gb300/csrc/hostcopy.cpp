// Host copy pool: see hostcopy.h.
#include "hostcopy.h"

#include <algorithm>
#include <cstring>

namespace olap {

namespace {
constexpr size_t MIN_PIECE = 1u << 20;   // below this a piece is not worth a thread
}

HostCopyPool::HostCopyPool(int helpers) {
    for (int i = 0; i < helpers; ++i) threads_.emplace_back([this, i] { work(i); });
}

HostCopyPool::~HostCopyPool() {
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
    }
    go_.notify_all();
    for (std::thread& t : threads_) t.join();
}

// Take pieces until none is left; called by the caller and the helpers.
void HostCopyPool::run_pieces() {
    while (true) {
        size_t i;
        {
            std::lock_guard<std::mutex> g(mu_);
            if (next_ >= pieces_) return;
            i = next_++;
        }
        const size_t off = i * piece_;
        std::memcpy(dst_ + off, src_ + off, std::min(piece_, bytes_ - off));
        bool all = false;
        {
            std::lock_guard<std::mutex> g(mu_);
            all = ++finished_ == pieces_;
        }
        if (all) done_.notify_all();
    }
}

void HostCopyPool::work(int) {
    unsigned long long seen = 0;
    while (true) {
        {
            std::unique_lock<std::mutex> lk(mu_);
            go_.wait(lk, [&] { return stop_ || gen_ != seen; });
            if (stop_) return;
            seen = gen_;
        }
        run_pieces();
    }
}

void HostCopyPool::copy(void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return;
    const size_t workers = threads_.size() + 1;
    if (threads_.empty() || bytes < 2 * MIN_PIECE) {
        std::memcpy(dst, src, bytes);
        return;
    }
    // Pieces of at least MIN_PIECE, a multiple of 4 KiB, about two per worker.
    size_t piece = std::max(MIN_PIECE, (bytes / (2 * workers) + 4095) & ~static_cast<size_t>(4095));
    {
        std::lock_guard<std::mutex> g(mu_);
        dst_ = static_cast<unsigned char*>(dst);
        src_ = static_cast<const unsigned char*>(src);
        bytes_ = bytes;
        piece_ = piece;
        pieces_ = (bytes + piece - 1) / piece;
        next_ = 0;
        finished_ = 0;
        ++gen_;
    }
    go_.notify_all();
    run_pieces();
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return finished_ == pieces_; });
}

}  // namespace olap
