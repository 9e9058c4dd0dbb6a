// fhp_arena.h -- first-fit offset allocator over one device buffer.
//
// A batch of lattices lives in one device allocation (the "arena"); members
// join and leave while others keep running, so their plane buffers are carved
// out of the arena by this allocator instead of one cudaMalloc each.  It only
// manages offsets (host-side bookkeeping), never touches device memory, and
// has no CUDA dependency, so it can be unit-tested on the CPU.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace fhp {

class Arena {
public:
    static constexpr size_t kAlign = 256;

    Arena() = default;
    explicit Arena(size_t bytes) { reset(bytes); }

    void reset(size_t bytes) {
        capacity_ = bytes / kAlign * kAlign;
        free_.clear();
        used_ = 0;
        if (capacity_) free_[0] = capacity_;
    }

    // Offset of a new block of at least `bytes` (rounded up to kAlign), or
    // SIZE_MAX if no free range is large enough.  First fit by address.
    size_t allocate(size_t bytes) {
        const size_t need = round(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t off = it->first;
            const size_t rest = it->second - need;
            free_.erase(it);
            if (rest) free_[off + need] = rest;
            used_ += need;
            return off;
        }
        return SIZE_MAX;
    }

    // Return the block [off, off + bytes) (bytes as passed to allocate);
    // merges with free neighbours.  Returns false for an invalid block.
    bool release(size_t off, size_t bytes) {
        const size_t size = round(bytes ? bytes : 1);
        if (off % kAlign || off + size > capacity_) return false;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first < off + size) return false;          // overlaps a free range
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second > off) return false;                      // overlaps a free range
        }
        size_t start = off, len = size;
        if (next != free_.end() && next->first == off + size) {                      // merge right
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {                                 // merge left
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
        used_ -= size;
        return true;
    }

    size_t capacity() const { return capacity_; }
    size_t used() const { return used_; }
    size_t free_bytes() const { return capacity_ - used_; }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }
    size_t free_ranges() const { return free_.size(); }

    static size_t round(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

private:
    size_t capacity_ = 0;
    size_t used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length of each free range
};

}  // namespace fhp
