"""Host logic of the serving loop's arena allocator (paper_1511_08463_gb300/csrc/arena.hpp),
compiled with g++ and driven by a seeded random sequence of allocations and frees, checked
against a first-fit reference model: identical offsets, alignment, no overlap, coalescing back
to one block, peak tracking.  No GPU."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1511_08463_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "arena.hpp"
int main() {
  pf::ArenaAlloc a;
  char op;
  unsigned long long x, y;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'i') { std::scanf("%llu", &x); a.init(x); }
    else if (op == 'a') {
      std::scanf("%llu", &x);
      size_t off = 0;
      bool ok = a.alloc(x, &off);
      std::printf("%lld\n", ok ? (long long)off : -1LL);
    } else if (op == 'f') { std::scanf("%llu %llu", &x, &y); a.release(x, y); }
    else if (op == 's') {
      std::printf("%zu %zu %zu %zu %zu\n", a.size(), a.used(), a.peak(), a.free_blocks(),
                  a.largest_free());
    }
  }
  return 0;
}
"""

ALIGN = 256


def _round(n):
    n = (n + ALIGN - 1) // ALIGN * ALIGN
    return n if n else ALIGN


class FirstFit:
    def __init__(self, size):
        self.size = size // ALIGN * ALIGN
        self.free = [(0, self.size)] if self.size else []
        self.used = self.peak = 0

    def alloc(self, n):
        n = _round(n)
        for k, (o, ln) in enumerate(self.free):
            if ln >= n:
                self.free[k:k + 1] = [(o + n, ln - n)] if ln > n else []
                self.used += n
                self.peak = max(self.peak, self.used)
                return o
        return -1

    def release(self, off, n):
        n = _round(n)
        self.used -= n
        blocks = sorted(self.free + [(off, n)])
        merged = []
        for o, ln in blocks:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("arena")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_first_fit_matches_reference(driver, seed):
    rng = random.Random(seed)
    size = rng.choice([1 << 20, 3 * (1 << 20) + 100, 10_000_000])
    ref = FirstFit(size)
    cmds, expect, live = [f"i {size}"], [], []
    for _ in range(400):
        if live and rng.random() < 0.45:
            off, n = live.pop(rng.randrange(len(live)))
            cmds.append(f"f {off} {n}")
            ref.release(off, n)
        else:
            n = rng.choice([1, 255, 256, 257, rng.randrange(1, 300_000)])
            o = ref.alloc(n)
            cmds.append(f"a {n}")
            expect.append(o)
            if o >= 0:
                live.append((o, n))
                # offsets aligned, inside the arena, no overlap with other live blocks
                assert o % ALIGN == 0 and o + _round(n) <= ref.size
                for (o2, n2) in live[:-1]:
                    assert o + _round(n) <= o2 or o2 + _round(n2) <= o
    for off, n in live:
        cmds.append(f"f {off} {n}")
        ref.release(off, n)
    cmds.append("s")
    out = subprocess.run([driver], input="\n".join(cmds) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    got = [int(v) for v in out[:len(expect)]]
    assert got == expect
    size_c, used, peak, nfree, largest = map(int, out[len(expect)].split())
    assert size_c == ref.size and used == 0 and peak == ref.peak
    assert nfree == 1 and largest == ref.size  # everything freed: one coalesced block
