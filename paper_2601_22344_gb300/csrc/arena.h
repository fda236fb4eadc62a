// First-fit allocator over one fixed region (offsets only; the region itself
// is allocated once by the serving session).  Blocks are 256-byte aligned;
// freed blocks are merged with free neighbours.  Plain host C++ (no CUDA), so
// it is tested on the CPU (tests/test_arena.py).
#pragma once

#include <stdint.h>

#include <iterator>
#include <map>

namespace rplu {

class Arena {
 public:
  static constexpr int64_t kAlign = 256;

  explicit Arena(int64_t size = 0) { reset(size); }

  void reset(int64_t size) {
    size_ = size / kAlign * kAlign;
    free_.clear();
    if (size_ > 0) free_[0] = size_;
    used_ = 0;
  }

  // Offset of a block of at least `bytes`, or -1 when no free block is large enough.
  int64_t alloc(int64_t bytes) {
    const int64_t need = round_up(bytes > 0 ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const int64_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > need) free_[off + need] = len - need;
      used_ += need;
      return off;
    }
    return -1;
  }

  // Returns a block obtained from alloc(bytes) with the same `bytes`.
  void release(int64_t off, int64_t bytes) {
    const int64_t len = round_up(bytes > 0 ? bytes : 1);
    used_ -= len;
    auto next = free_.lower_bound(off);
    int64_t start = off, end = off + len;
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        free_.erase(prev);
      }
    }
    if (next != free_.end() && next->first == end) {
      end = next->first + next->second;
      free_.erase(next);
    }
    free_[start] = end - start;
  }

  int64_t size() const { return size_; }
  int64_t used() const { return used_; }
  int64_t largest_free() const {
    int64_t m = 0;
    for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }
  int64_t free_blocks() const { return (int64_t)free_.size(); }

  static int64_t round_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

 private:
  int64_t size_ = 0;
  int64_t used_ = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length
};

}  // namespace rplu
