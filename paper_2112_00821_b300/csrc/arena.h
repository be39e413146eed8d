// Host-side allocator of the serving form's device reservation: offsets into
// one block, bookkeeping only, so allocating and freeing never touch the
// device.  Plain C++ (no CUDA), tested on the CPU.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>
#include <unordered_map>

namespace fmh {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Best-fit allocator over one block of `cap` bytes at `base` (256-byte
// granules).
class Arena {
public:
    bool init(size_t cap, void* base)
    {
        base_ = static_cast<unsigned char*>(base);
        cap = cap & ~(kAlign - 1);           // whole granules: every block stays 256-byte aligned
        cap_ = cap;
        free_.clear();
        live_.clear();
        if (cap) free_[0] = cap;
        used_ = peak_ = 0;
        return true;
    }
    // offset of a block of `bytes`, or SIZE_MAX when nothing fits: best fit
    // from the low end, or (high) carved from the end of the highest free
    // block, so that small long-lived blocks (frames) gather at the top and
    // the request scratch keeps the large free space at the bottom
    size_t alloc(size_t bytes, bool high = false)
    {
        bytes = align_up(bytes ? bytes : 1);
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            if (best == free_.end() || (high ? it->first > best->first : it->second < best->second)) best = it;
        }
        if (best == free_.end()) return SIZE_MAX;
        const size_t off = best->first, sz = best->second;
        free_.erase(best);
        size_t at = off;
        if (high) {
            at = off + sz - bytes;
            if (sz > bytes) free_[off] = sz - bytes;
        } else if (sz > bytes) {
            free_[off + bytes] = sz - bytes;
        }
        live_[at] = bytes;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return at;
    }
    void release(size_t off)
    {
        auto it = live_.find(off);
        if (it == live_.end()) return;
        size_t sz = it->second;
        live_.erase(it);
        used_ -= sz;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + sz == nx->first) { sz += nx->second; nx = free_.erase(nx); }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) { pv->second += sz; return; }
        }
        free_[off] = sz;
    }
    unsigned char* at(size_t off) const { return base_ + off; }
    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    unsigned char* base_ = nullptr;
    size_t cap_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
    std::unordered_map<size_t, size_t> live_;
};

}  // namespace fmh
