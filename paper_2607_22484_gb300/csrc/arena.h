// First-fit range allocator over [0, size) in `align`-byte units: the serving loop's
// placement of each admitted request's workspace inside the context's workspace. Pure
// host code, checked on the host by the tests.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace svt {

struct Arena {
    size_t size = 0;
    size_t align = 256;
    std::map<size_t, size_t> free_;  // offset -> length of each free range, disjoint, coalesced
    static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
    void reset(size_t s)
    {
        size = s;
        free_.clear();
        if (s)
            free_[0] = s;
    }
    // The lowest free range that fits `len` (rounded up to the alignment); false if none.
    bool alloc(size_t len, size_t *off)
    {
        len = round_up(len, align);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                size_t rest = it->second - len;
                size_t roff = it->first + len;
                free_.erase(it);
                if (rest)
                    free_[roff] = rest;
                return true;
            }
        }
        return false;
    }
    // Return a range given by alloc (same length); it merges with free neighbours.
    void release(size_t off, size_t len)
    {
        len = round_up(len, align);
        auto it = free_.emplace(off, len).first;
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
};

} // namespace svt
