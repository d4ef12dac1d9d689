// ci_arena.h -- sub-allocator of the serving loop's arena (ci_server.cu).
// Host-only C++ (no CUDA): offsets into the caller's device arena in 256-byte
// units, first fit from the bottom for request outputs, highest fit for stream
// states, neighbours coalesced on release.  Kept in its own header so its
// invariants are tested on the CPU (tests/test_arena_cpu.py).
#pragma once

#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>

namespace ci {

inline uint64_t round256(uint64_t b) { return (b + 255ull) & ~255ull; }

// Sub-allocator over the caller's arena (offsets, 256-byte units): first fit
// from the bottom for outputs, highest fit for stream states; neighbours
// coalesce on release.
class Arena {
   public:
    void init(uint64_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
        used_ = peak_ = 0;
    }
    bool alloc(uint64_t bytes, uint64_t *off) {
        bytes = round256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const uint64_t o = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[o + bytes] = rem;
            *off = o;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    // Highest-addressed fit, taken from the top end of its free block.  Stream
    // states (small, long-lived) come from the top of the arena and outputs
    // from the bottom, so states do not fragment the space outputs need.
    bool alloc_high(uint64_t bytes, uint64_t *off) {
        bytes = round256(bytes);
        for (auto it = free_.rbegin(); it != free_.rend(); ++it) {
            if (it->second < bytes) continue;
            it->second -= bytes;
            *off = it->first + it->second;
            if (it->second == 0) free_.erase(std::next(it).base());
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = round256(bytes);
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
    uint64_t size() const { return size_; }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }
    // Visits the free blocks (offset, bytes) in address order.
    template <class F>
    void for_each_free(F f) const {
        for (const auto &kv : free_) f(kv.first, kv.second);
    }

   private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t size_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace ci
