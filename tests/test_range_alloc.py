"""The first-fit range allocator behind the batch pool and the serving
arenas (`csrc/range_alloc.h`), host logic checked on the CPU: a small C++
driver runs random alloc / release sequences and every answer is compared
with a plain Python model; live ranges never overlap and frees coalesce."""
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1206_0919_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "range_alloc.h"
int main() {
  long long cap, align;
  if (std::scanf("%lld %lld", &cap, &align) != 2) return 1;
  shasta::RangeAlloc a(align);
  a.reset(cap);
  char op;
  long long x, y;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'a' && std::scanf("%lld", &x) == 1) std::printf("%lld\n", a.alloc(x));
    else if (op == 'r' && std::scanf("%lld %lld", &x, &y) == 2) a.release(x, y);
    else if (op == 'l') std::printf("%lld\n", a.largest());
  }
  return 0;
}
"""


class Model:
    """First fit over free ranges sorted by start; lengths rounded up to the
    alignment; a release merges with free neighbours."""

    def __init__(self, cap, align):
        self.align = align
        self.free = [[0, cap]] if cap > 0 else []

    def rounded(self, n):
        return (n + self.align - 1) // self.align * self.align

    def alloc(self, n):
        n = self.rounded(n)
        for i, (s, length) in enumerate(self.free):
            if length >= n:
                if length == n:
                    del self.free[i]
                else:
                    self.free[i] = [s + n, length - n]
                return s
        return -1

    def release(self, s, n):
        n = self.rounded(n)
        self.free.append([s, n])
        self.free.sort()
        merged = []
        for a, b in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1][1] += b
            else:
                merged.append([a, b])
        self.free = merged

    def largest(self):
        return max((b for _, b in self.free), default=0)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("ra")
    src = d / "ra.cpp"
    src.write_text(DRIVER)
    exe = d / "ra"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("align", [1, 32, 256])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_sequences(driver, align, seed):
    rng = random.Random(seed * 10 + align)
    cap = 64 * 1024
    model = Model(cap, align)
    ops, expect, live = [], [], []
    # the script is fixed in advance from the model's answers
    for _ in range(3000):
        if live and rng.random() < 0.45:
            s, n = live.pop(rng.randrange(len(live)))
            ops.append(f"r {s} {n}")
            model.release(s, n)
        else:
            n = rng.randint(1, 3000)
            ops.append(f"a {n}")
            s = model.alloc(n)
            expect.append(s)
            if s >= 0:
                live.append((s, n))
        ops.append("l")
        expect.append(model.largest())
    out = subprocess.run([driver], input=f"{cap} {align}\n" + "\n".join(ops) + "\n",
                         capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == expect
    # live ranges are disjoint, inside the capacity, aligned
    spans = sorted((s, s + model.rounded(n)) for s, n in live)
    for (a0, a1), (b0, _) in zip(spans, spans[1:]):
        assert a1 <= b0
    assert all(0 <= s and e <= cap and s % align == 0 for s, e in spans)


def test_coalescing_returns_the_whole_range(driver):
    """Freeing every block in any order leaves one free range of the full
    capacity."""
    ops = ["a 100", "a 200", "a 300", "a 400", "r 100 200", "r 0 100", "r 600 400",
           "r 300 300", "l", "a 1000"]
    out = subprocess.run([driver], input="1000 1\n" + "\n".join(ops) + "\n",
                         capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [0, 100, 300, 600, 1000, 0]
