"""The host's cuts of a sweep's work into ranges (`csrc/work_ranges.h`),
checked on the CPU: a small C++ driver prints the bounds for a set of line
lengths, range counts and CTA-rank weights, and every answer is checked for
what the kernels rely on (the bounds cover the work once, in order; on the x
path a bound inside a line falls on an 8-cell chunk boundary; no more ranges
than asked for) and for what the cut is for (about equal streaming cost per
unit of weight, with more work for the CTAs launched first on an SM)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1206_0919_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "work_ranges.h"
int main() {
  long long total, n, R, align, sms, K, wpb;
  double halo, edge, skew;
  while (std::scanf("%lld %lld %lld %lld %lf %lf %lld %lld %lld %lf", &total, &n, &R, &align,
                    &halo, &edge, &sms, &K, &wpb, &skew) == 10) {
    auto w = [&](long long r) { return shasta::rank_weight(r, sms, K, wpb, skew); };
    const std::vector<int> b = shasta::balanced_bounds(total, n, R, align, halo, edge, w);
    std::printf("%zu", b.size());
    for (int x : b) std::printf(" %d", x);
    std::printf("\n");
  }
  return 0;
}
"""

HALO, EDGE, MIN_PIECE = 13.0, 11.0, 8


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("wr")
    src, exe = d / "wr.cpp", d / "wr"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def weight(r, sms, K, wpb, skew):
    if K < 2:
        return 1.0
    rank = (r % (sms * K * wpb)) // wpb // sms
    return 1.0 + skew * (1.0 - 2.0 * rank / (K - 1))


def cost(x, e, n):
    """Streaming cost of range [x, e): per piece its positions, the halo and
    the line ends it touches."""
    c, y = 0.0, x
    while y < e:
        line_end = (y // n + 1) * n
        t = min(line_end, e) - y
        c += t + HALO + (EDGE if y % n == 0 else 0.0) + (EDGE if y + t == line_end else 0.0)
        y += t
    return c


# (total, n, R, align, sms, K, wpb, skew): the single-event work of 200^3 and
# 256^3 (x and y/z paths, one range per resident warp), ragged and tiny cases
CASES = [
    (1250 * 200, 200, 1812, 8, 152, 3, 4, 0.0),
    (1250 * 200, 200, 1812, 1, 152, 3, 4, 0.0),
    (1250 * 200, 200, 1812, 8, 152, 3, 4, 0.04),
    (1250 * 200, 200, 1812, 1, 152, 3, 4, 0.08),
    (2048 * 256, 256, 1821, 8, 152, 3, 4, 0.04),
    (2048 * 256, 256, 1821, 1, 152, 3, 4, 0.08),
    (2048 * 256, 256, 3642, 1, 152, 3, 4, 0.04),  # two ranges per warp
    (425 * 77, 77, 1000, 8, 152, 3, 4, 0.04),
    (13 * 37, 37, 50, 1, 152, 3, 4, 0.0),
    (3 * 21, 21, 500, 8, 4, 3, 4, 0.08),  # more ranges asked for than chunks exist
    (5 * 9, 9, 1, 1, 152, 3, 4, 0.0),  # one range: the whole work
    (64 * 64, 64, 32, 8, 4, 1, 4, 0.08),  # one CTA per SM: no skew
]


def run(driver, cases):
    inp = "".join(f"{t} {n} {R} {a} {HALO} {EDGE} {s} {K} {w} {sk}\n"
                  for t, n, R, a, s, K, w, sk in cases)
    out = subprocess.run([driver], input=inp, capture_output=True, text=True, check=True).stdout
    res = []
    for line in out.strip().splitlines():
        v = [int(x) for x in line.split()]
        assert v[0] == len(v) - 1
        res.append(v[1:])
    return res


def test_bounds_cover_the_work_in_order(driver):
    for case, b in zip(CASES, run(driver, CASES)):
        total, n, R, align = case[:4]
        assert b[0] == 0 and b[-1] == total, case
        assert all(x < y for x, y in zip(b, b[1:])), case
        assert len(b) - 1 <= max(R, 1) or len(b) - 1 <= -(-total // align), case
        for x in b[1:-1]:
            # the x path moves data in 8-cell chunks of a line
            assert (x % n) % align == 0, (case, x)


def test_costs_balanced_per_unit_of_weight(driver):
    for case, b in zip(CASES, run(driver, CASES)):
        total, n, R, align, sms, K, wpb, skew = case
        nr = len(b) - 1
        if nr < 4:
            continue
        c = [cost(b[r], b[r + 1], n) for r in range(nr)]
        w = [weight(r, sms, K, wpb, skew) for r in range(nr)]
        per = [ci / wi for ci, wi in zip(c, w)]
        fair = sum(c) / sum(w)
        # a range overshoots its share by at most what one cut can add: a
        # chunk, a sliver of a line, a piece's halo and two line ends
        slack = align + MIN_PIECE + HALO + 2 * EDGE
        assert max(per) <= fair + slack / min(w), (case, max(per), fair)


def test_first_ctas_of_an_sm_take_more_work(driver):
    cases = [(1250 * 200, 200, 1812, 1, 152, 3, 4, s) for s in (0.0, 0.08)]
    for (total, n, R, align, sms, K, wpb, skew), b in zip(cases, run(driver, cases)):
        by_rank = [[], [], []]
        for r in range(len(b) - 1):
            rank = (r % (sms * K * wpb)) // wpb // sms
            by_rank[rank].append(cost(b[r], b[r + 1], n))
        mean = [sum(v) / len(v) for v in by_rank]
        if skew == 0.0:
            assert max(mean) - min(mean) < 0.02 * mean[1], mean
        else:
            assert mean[0] > 1.05 * mean[1] > 1.05 * mean[2], mean
