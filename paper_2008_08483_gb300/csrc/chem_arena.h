// chem_arena.h -- first-fit allocator of offsets inside one fixed block (the serving loop's
// HBM budget and its page-locked host mirror).  Host code only, no CUDA: blocks are carved
// first-fit from a sorted free list and coalesced with their neighbours on release.
#pragma once

#include <stddef.h>

#include <algorithm>
#include <iterator>
#include <map>

namespace chem {

// First-fit allocator over [0, size): offsets only; the bytes live elsewhere.
struct Arena {
    size_t size = 0, in_use = 0, peak = 0;
    std::map<size_t, size_t> free_;   // offset -> length, disjoint and coalesced

    void init(size_t n)
    {
        size = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    size_t largest_free() const
    {
        size_t b = 0;
        for (auto &kv : free_) b = std::max(b, kv.second);
        return b;
    }
    bool alloc(size_t bytes, size_t &off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            off = it->first;
            const size_t rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            in_use += bytes;
            peak = std::max(peak, in_use);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        in_use -= bytes;
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
};

}  // namespace chem
