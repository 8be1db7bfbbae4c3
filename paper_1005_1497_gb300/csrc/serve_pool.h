// serve_pool.h -- the convolution server's device-memory pool: first-fit
// allocation over one region of byte offsets, 256-byte granules, with
// coalescing of free blocks on release.  Host-only bookkeeping (no CUDA).
#pragma once

#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace ntt {

// First-fit allocator over one device region, with coalescing of free blocks.
class Pool {
  public:
    void init(size_t bytes) { free_.clear(); free_[0] = bytes; size_ = bytes; used_ = peak_ = 0; }
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t peak() const { return peak_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace ntt
