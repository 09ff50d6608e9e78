// work_ranges.h -- host-side cuts of a sweep's work into ranges of about
// equal streaming cost (FP32 / MIXED single-event sweeps).  Host code only.
#pragma once

#include <algorithm>
#include <vector>

namespace shasta {

// Bounds of at most R contiguous work ranges over `total` positions (lines
// of n positions, one after the other) with streaming costs in proportion to
// weight(r): a piece (the part of a range within one line) costs its
// positions plus `halo` positions of lead-in and lag plus `edge` for each
// line end it touches, so a range that crosses or reaches a line end is
// shorter.  Bounds inside a line fall on multiples of `align`; a range takes
// no further piece shorter than 8 positions.  The smallest cost scale T that
// needs at most R ranges is found by bisection.
template <class Weight>
inline std::vector<int> balanced_bounds(long long total, long long n, long long R,
                                        long long align, double halo, double edge,
                                        Weight weight) {
  const long long kMinPiece = 8;
  auto cut = [&](double T, std::vector<int>* out) -> long long {
    long long x = 0, count = 0;
    if (out) out->assign(1, 0);
    while (x < total) {
      double budget = T * weight(count);
      long long y = x;
      while (y < total) {
        const long long line_end = (y / n + 1) * n;
        const double fixed = halo + (y == line_end - n ? edge : 0.0);
        if (budget <= fixed) break;
        long long take;
        if ((double)(line_end - y) + fixed + edge <= budget) {
          take = line_end - y;  // the rest of the line, its end included
        } else {
          take = std::min(line_end - y - 1, (long long)(budget - fixed));
          const long long e = y + take;
          take -= (e - (e / n) * n) % align;  // end on a chunk boundary of the line
          if (line_end - (y + take) < kMinPiece) take = line_end - y;  // no sliver left over
        }
        if (take <= 0 || (y != x && take < kMinPiece && y + take < line_end)) break;
        budget -= (double)take + fixed + (y + take == line_end ? edge : 0.0);
        y += take;
      }
      if (y == x) y = std::min((x / n + 1) * n, x + align);  // at least one chunk
      ++count;
      x = y;
      if (out) out->push_back((int)y);
    }
    return count;
  };
  double lo = 0.0, hi = 2.0 * ((double)total + (halo + 2.0 * edge) * (double)(total / n + 2)) + 1.0;
  for (int it = 0; it < 64 && hi - lo > 1e-3; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (cut(mid, nullptr) <= R)
      hi = mid;
    else
      lo = mid;
  }
  std::vector<int> b;
  cut(hi, &b);
  return b;
}

// Work share of range r in a launch of K CTAs of wpb warps per SM on `sms`
// SMs: range r runs on warp r mod (sms K wpb), whose block b = warp / wpb is
// the (b / sms)-th CTA of its SM when blocks are handed to the SMs in order;
// the first CTA of an SM takes 1 + skew, the last 1 - skew.
inline double rank_weight(long long r, long long sms, long long K, long long wpb, double skew) {
  if (K < 2 || sms < 1 || wpb < 1) return 1.0;
  const long long W = sms * K * wpb;
  const long long rank = (r % W) / wpb / sms;
  return 1.0 + skew * (1.0 - 2.0 * (double)rank / (double)(K - 1));
}

}  // namespace shasta
