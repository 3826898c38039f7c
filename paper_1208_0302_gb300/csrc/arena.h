// First-fit arena allocator over a fixed byte range (host-side bookkeeping for
// the serving loop's device and pinned-host arenas).  Offsets are aligned to
// `align` bytes; freed ranges coalesce with their neighbours.  Not
// thread-safe: the caller holds its own lock.
#pragma once

#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace genesis {

class Arena {
  public:
    static constexpr size_t kNone = ~(size_t)0;

    explicit Arena(size_t bytes = 0, size_t align = 256) : size_(bytes), align_(align)
    {
        if (bytes) free_[0] = bytes;
    }

    size_t size() const { return size_; }
    size_t used() const { return used_; }

    static size_t round_up(size_t n, size_t a) { return (n + a - 1) / a * a; }

    // Offset of a block of at least `bytes`, or kNone if no free range fits.
    size_t alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 1;
        const size_t need = round_up(bytes, align_);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= need) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > need) free_[off + need] = len - need;
                live_[off] = need;
                used_ += need;
                return off;
            }
        }
        return kNone;
    }

    // Returns false if off is not a live block.
    bool release(size_t off)
    {
        auto lv = live_.find(off);
        if (lv == live_.end()) return false;
        size_t start = off, len = lv->second;
        used_ -= len;
        live_.erase(lv);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && start + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
        return true;
    }

    // Consistency: free and live ranges tile [0, size) without overlap.
    bool check() const
    {
        std::map<size_t, size_t> all(free_);
        for (const auto &kv : live_) {
            if (all.count(kv.first)) return false;
            all[kv.first] = kv.second;
        }
        size_t at = 0, live = 0;
        for (const auto &kv : all) {
            if (kv.first != at) return false;
            at += kv.second;
        }
        for (const auto &kv : live_) live += kv.second;
        // adjacent free ranges must have been merged
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            auto nx = std::next(it);
            if (nx != free_.end() && it->first + it->second == nx->first) return false;
        }
        return at == size_ && live == used_;
    }

    size_t largest_free() const
    {
        size_t m = 0;
        for (const auto &kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

  private:
    size_t size_, align_, used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    std::map<size_t, size_t> live_;  // offset -> length
};

}  // namespace genesis
