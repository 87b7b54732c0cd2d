// First-fit allocator of the serving engine's output arena: [0, size) bytes
// handed out in multiples of a granule, the free space kept as a map from
// offset to length so that a release merges with its free neighbours, and
// the free lengths in a multiset so that a request larger than every free
// block fails without a scan.
// Host-only (no CUDA), so it is tested on the CPU by itself.
#pragma once

#include <stdint.h>

#include <iterator>
#include <map>
#include <set>

namespace gbrng {

class Arena {
public:
    Arena(uint64_t size, uint64_t granule)
        : granule_(granule), size_(size / granule * granule)
    {
        if (size_)
            add(0, size_);
    }
    // The lowest free offset with room for `bytes` (rounded up to the
    // granule); false when no free block is large enough.
    bool alloc(uint64_t bytes, uint64_t *off)
    {
        bytes = round_up(bytes);
        if (bytes > largest())
            return false;  // no block is large enough: no scan
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes;
                const uint64_t at = it->first + bytes;
                erase(it);
                if (rest)
                    add(at, rest);
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    // Returns [off, off + bytes) (bytes rounded up as in alloc) to the free
    // space, merged with the free blocks that touch it.
    void release(uint64_t off, uint64_t bytes)
    {
        bytes = round_up(bytes);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                const uint64_t at = prev->first, merged = prev->second + bytes;
                erase(prev);
                add(at, merged);
                return;
            }
        }
        add(off, bytes);
    }
    // The largest free block (0 when none).
    uint64_t largest() const { return sizes_.empty() ? 0 : *sizes_.rbegin(); }
    uint64_t used() const { return used_; }
    uint64_t size() const { return size_; }
    size_t free_blocks() const { return free_.size(); }

private:
    uint64_t round_up(uint64_t bytes) const
    {
        return (bytes + granule_ - 1) / granule_ * granule_;
    }
    void add(uint64_t off, uint64_t len)
    {
        free_[off] = len;
        sizes_.insert(len);
    }
    std::map<uint64_t, uint64_t>::iterator erase(std::map<uint64_t, uint64_t>::iterator it)
    {
        sizes_.erase(sizes_.find(it->second));
        return free_.erase(it);
    }
    uint64_t granule_;
    uint64_t size_;
    uint64_t used_ = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> length
    std::multiset<uint64_t> sizes_;       // the lengths of the free blocks
};

}  // namespace gbrng
