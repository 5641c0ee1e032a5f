// First-fit allocator of offsets in a device arena (host-side bookkeeping only), used by the
// serving loop to place each admitted job's workspace.  Blocks are 256-byte aligned; freed blocks
// coalesce with free neighbours, so an arena that empties is again one free block.  Not
// thread-safe (the serving loop holds its lock around every call).
#pragma once
#include <stddef.h>

#include <algorithm>
#include <iterator>
#include <map>

namespace pf {

constexpr size_t ARENA_ALIGN = 256;

inline size_t round_up(size_t n) { return (n + ARENA_ALIGN - 1) / ARENA_ALIGN * ARENA_ALIGN; }

class ArenaAlloc {
 public:
  // the arena is [0, size); size is rounded down to the alignment
  void init(size_t size) {
    size = size / ARENA_ALIGN * ARENA_ALIGN;
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
    used_ = peak_ = 0;
  }
  // first free block that holds round_up(n) bytes; false if none (nothing changes)
  bool alloc(size_t n, size_t* off) {
    n = round_up(n);
    if (n == 0) n = ARENA_ALIGN;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t o = it->first, rem = it->second - n;
      free_.erase(it);
      if (rem) free_[o + n] = rem;
      *off = o;
      used_ += n;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  // give back a block returned by alloc(n) at offset off
  void release(size_t off, size_t n) {
    n = round_up(n);
    if (n == 0) n = ARENA_ALIGN;
    used_ -= n;
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
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t free_blocks() const { return free_.size(); }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  std::map<size_t, size_t> free_;  // offset -> length of each free block
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace pf
