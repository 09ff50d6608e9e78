// range_alloc.h -- first-fit allocator of ranges [0, cap) of some unit
// (cells of a state pool, bytes of a staging arena), with coalescing frees.
#pragma once

#include <algorithm>
#include <iterator>
#include <map>

namespace shasta {

class RangeAlloc {
 public:
  explicit RangeAlloc(long long align = 1) : align_(align > 0 ? align : 1) {}
  void reset(long long cap) {
    free_.clear();
    if (cap > 0) free_[0] = cap;
  }
  long long rounded(long long len) const { return (len + align_ - 1) / align_ * align_; }
  // Start of a free range of len units (rounded up to the alignment), or -1.
  long long alloc(long long len) {
    len = rounded(len);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= len) {
        const long long start = it->first, rest = it->second - len;
        free_.erase(it);
        if (rest > 0) free_[start + len] = rest;
        return start;
      }
    }
    return -1;
  }
  void release(long long start, long long len) {
    len = rounded(len);
    auto nx = free_.lower_bound(start);
    if (nx != free_.end() && start + len == nx->first) {
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == start) {
        pv->second += len;
        return;
      }
    }
    free_[start] = len;
  }
  long long largest() const {
    long long m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  long long align_;
  std::map<long long, long long> free_;
};

}  // namespace shasta
