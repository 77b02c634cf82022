// bcn_pool.h -- host-side sub-allocator for a device output pool.
//
// The serving loop owns one device allocation (the output pool) and places
// each admitted request's output inside it.  This allocator only does the
// bookkeeping on the host: it hands out aligned byte ranges [off, off+size)
// of a pool of `capacity` bytes, first fit over an address-ordered free list,
// and merges neighbouring free ranges on release, so a request is admitted
// exactly when a large enough range is free.  It never touches the device.
#pragma once
#include <cstdint>
#include <iterator>
#include <map>

namespace bcn {

struct Pool {
  uint64_t capacity;
  uint64_t align;
  uint64_t in_use = 0;
  uint64_t peak = 0;
  uint64_t live = 0;
  std::map<uint64_t, uint64_t> free_by_off;  // offset -> size, address ordered
  std::map<uint64_t, uint64_t> used_by_off;  // offset -> size

  Pool(uint64_t cap, uint64_t al) : capacity(cap), align(al) {
    if (cap) free_by_off.emplace(0, cap);
  }

  bool alloc(uint64_t bytes, uint64_t* off) {
    if (bytes == 0) bytes = 1;
    if (bytes > capacity) return false;  // also keeps the rounding below from wrapping
    const uint64_t need = bytes + (align - bytes % align) % align;
    if (need < bytes) return false;
    for (auto it = free_by_off.begin(); it != free_by_off.end(); ++it) {
      if (it->second >= need) {
        const uint64_t o = it->first, sz = it->second;
        free_by_off.erase(it);
        if (sz > need) free_by_off.emplace(o + need, sz - need);
        used_by_off.emplace(o, need);
        in_use += need;
        live += 1;
        if (in_use > peak) peak = in_use;
        *off = o;
        return true;
      }
    }
    return false;
  }

  bool release(uint64_t off) {
    auto u = used_by_off.find(off);
    if (u == used_by_off.end()) return false;
    uint64_t o = u->first, sz = u->second;
    used_by_off.erase(u);
    in_use -= sz;
    live -= 1;
    auto next = free_by_off.lower_bound(o);
    if (next != free_by_off.end() && o + sz == next->first) {  // merge with the right
      sz += next->second;
      next = free_by_off.erase(next);
    }
    if (next != free_by_off.begin()) {  // merge with the left
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        prev->second += sz;
        return true;
      }
    }
    free_by_off.emplace(o, sz);
    return true;
  }

  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& kv : free_by_off)
      if (kv.second > m) m = kv.second;
    return m;
  }
};

}  // namespace bcn
