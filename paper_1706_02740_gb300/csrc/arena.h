// First-fit bookkeeping of one contiguous device range (offsets only; no CUDA), used by the
// server to carve plans out of its memory budget.  Blocks are multiples of kArenaGrain bytes;
// freed blocks coalesce with free neighbours, so a range that is entirely free again is one block.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <iterator>
#include <map>

namespace sft {

constexpr size_t kArenaGrain = 256;

class OffsetArena {
 public:
  explicit OffsetArena(size_t capacity = 0) { reset(capacity); }

  void reset(size_t capacity) {
    cap_ = capacity / kArenaGrain * kArenaGrain;
    free_.clear();
    live_.clear();
    used_ = peak_ = 0;
    if (cap_) free_[0] = cap_;
  }

  // Offset of a new block of at least `bytes` (lowest fitting address), or -1 when none fits.
  int64_t alloc(size_t bytes) {
    const size_t n = (bytes + kArenaGrain - 1) / kArenaGrain * kArenaGrain;
    if (n == 0 || n > cap_) return -1;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, rest = it->second - n;
      free_.erase(it);
      if (rest) free_[off + n] = rest;
      live_[off] = n;
      used_ += n;
      if (used_ > peak_) peak_ = used_;
      return (int64_t)off;
    }
    return -1;
  }

  // Return a block; false if `off` is not the start of a live block.
  bool release(size_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return false;
    size_t n = it->second;
    live_.erase(it);
    used_ -= n;
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && off + n == nx->first) {   // merge with the next free block
      n += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {                         // and with the previous one
      auto pv = std::prev(nx);
      if (pv->first + pv->second == off) {
        start = pv->first;
        n += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = n;
    return true;
  }

  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t live_blocks() const { return live_.size(); }
  size_t free_blocks() const { return free_.size(); }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }

 private:
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;   // offset -> bytes
  std::map<size_t, size_t> live_;   // offset -> bytes
};

}  // namespace sft
