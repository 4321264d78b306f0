// First-fit allocator over one device buffer, by offsets in 256-byte granules
// (the serving runtime's admission by free HBM).  Host-only and independent
// of CUDA, so its logic is tested on the host against a brute-force model.
#pragma once

#include <stddef.h>

#include <algorithm>
#include <iterator>
#include <map>

namespace irk {

class PoolAllocator {
 public:
  static constexpr size_t kGranule = 256;

  // manage [0, bytes) rounded down to whole granules
  void init(size_t bytes) {
    size_ = bytes & ~(kGranule - 1);
    free_.clear();
    if (size_) free_[0] = size_;
    used_ = peak_ = 0;
  }
  // lowest-offset free block that fits `bytes` (rounded up to granules); false when none does
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(bytes);
    if (bytes == 0) bytes = kGranule;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  // return a block from alloc (same size argument); neighbours coalesce
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes);
    if (bytes == 0) bytes = kGranule;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  // the free list, in address order: (offset, bytes) of maximal free blocks
  const std::map<size_t, size_t>& free_blocks() const { return free_; }

 private:
  static size_t round_up(size_t b) { return (b + kGranule - 1) & ~(kGranule - 1); }
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace irk
