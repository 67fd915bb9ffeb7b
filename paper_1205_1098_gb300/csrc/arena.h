// First-fit allocator over the offsets [0, capacity) of a device arena, the
// serving runtime's memory budget.  Host code only (no CUDA), so it is also
// compiled into a CPU test harness.
#pragma once
#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace bto {

constexpr size_t kArenaGranule = 256;

// Free blocks are kept by offset and merged with their neighbours when
// released; every block is a multiple of 256 bytes.
class Arena {
 public:
    explicit Arena(size_t bytes) : cap_(bytes / kArenaGranule * kArenaGranule) {
        if (cap_) free_[0] = cap_;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = granules(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, start = it->first + bytes;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = granules(bytes);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t peak() const { return peak_; }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }
    size_t free_blocks() const { return free_.size(); }

 private:
    static size_t granules(size_t bytes) {
        bytes = std::max<size_t>(bytes, 1);
        return (bytes + kArenaGranule - 1) / kArenaGranule * kArenaGranule;
    }
    size_t cap_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace bto
