// arena.h -- first-fit allocator over one device region, by offset (the serving arena and its
// descriptor blob).  Host-only: no CUDA, so it is tested on the CPU.
#pragma once
#include <cstddef>
#include <iterator>
#include <map>

namespace swk {

// First-fit allocator over one device region (offsets; coalescing on release).
struct Arena {
    size_t bytes = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    void init(size_t n) {
        bytes = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(size_t n, size_t* off) {
        if (n == 0) { *off = 0; return true; }
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, o = it->first + n;
            free_.erase(it);
            if (rest) free_[o] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        if (n == 0) return;
        auto it = free_.emplace(off, n).first;
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

}  // namespace swk
