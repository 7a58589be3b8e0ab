// arena.h -- first-fit allocator of offsets inside one fixed device region.
//
// The serving loop admits a frame only when its images fit in a device arena of
// fixed size (admission by device memory).  This class does the bookkeeping on
// the host: it hands out aligned offsets, coalesces neighbouring free ranges on
// release and keeps the high-water mark.  It touches no device memory and no
// CUDA API, so it is plain C++ and is unit-tested on the CPU.
#pragma once

#include <stdint.h>

#include <iterator>
#include <map>

namespace ctm {

class Arena {
public:
    explicit Arena(int64_t size = 0, int64_t align = 256) { reset(size, align); }

    void reset(int64_t size, int64_t align)
    {
        align_ = align > 0 ? align : 1;
        size_ = size > 0 ? size / align_ * align_ : 0;
        free_.clear();
        live_.clear();
        used_ = peak_ = 0;
        if (size_ > 0) free_[0] = size_;
    }

    // Offset of a block of at least `bytes` (rounded up to the alignment), the
    // lowest free one that fits; -1 when none does.
    int64_t alloc(int64_t bytes)
    {
        if (bytes <= 0) bytes = 1;
        const int64_t need = (bytes + align_ - 1) / align_ * align_;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const int64_t off = it->first, rest = it->second - need;
            free_.erase(it);
            if (rest > 0) free_[off + need] = rest;
            live_[off] = need;
            used_ += need;
            if (used_ > peak_) peak_ = used_;
            return off;
        }
        return -1;
    }

    // Return a block obtained from alloc(); false if `off` is not a live block.
    bool release(int64_t off)
    {
        auto lv = live_.find(off);
        if (lv == live_.end()) return false;
        int64_t start = off, len = lv->second;
        used_ -= len;
        live_.erase(lv);
        auto nx = free_.lower_bound(start);
        if (nx != free_.end() && nx->first == start + len) {  // merge with the next range
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {  // merge with the previous range
            auto pv = std::prev(nx);
            if (pv->first + pv->second == start) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
        return true;
    }

    // Bytes a request of `bytes` occupies (its rounded size).
    int64_t rounded(int64_t bytes) const { return (bytes + align_ - 1) / align_ * align_; }
    int64_t size() const { return size_; }
    int64_t used() const { return used_; }
    int64_t peak() const { return peak_; }
    int64_t live_blocks() const { return (int64_t)live_.size(); }
    int64_t free_ranges() const { return (int64_t)free_.size(); }
    int64_t largest_free() const
    {
        int64_t m = 0;
        for (const auto &f : free_) m = f.second > m ? f.second : m;
        return m;
    }

private:
    int64_t size_ = 0, align_ = 256, used_ = 0, peak_ = 0;
    std::map<int64_t, int64_t> free_;  // offset -> length, disjoint and non-adjacent
    std::map<int64_t, int64_t> live_;  // offset -> length
};

}  // namespace ctm
