"""Host-side logic of the serving loop, without a GPU: the arena allocator
(paper_1208_0302_gb300/csrc/arena.h) under randomized alloc/free."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <random>
#include <vector>
#include "arena.h"
int main() {
    using genesis::Arena;
    std::mt19937_64 rng(12345);
    for (int trial = 0; trial < 50; ++trial) {
        const size_t size = 1 << (12 + trial % 10);
        Arena a(size, 256);
        std::vector<std::pair<size_t, size_t>> live;
        for (int step = 0; step < 4000; ++step) {
            if (live.empty() || rng() % 3) {
                const size_t n = 1 + rng() % (size / 4);
                const size_t off = a.alloc(n);
                if (off != Arena::kNone) {
                    if (off % 256 || off + n > size) return 1;
                    for (auto &l : live)
                        if (off < l.first + l.second && l.first < off + Arena::round_up(n, 256)) return 2;
                    live.push_back({off, Arena::round_up(n, 256)});
                } else if (a.largest_free() >= Arena::round_up(n, 256)) {
                    return 3;  // first fit must succeed when a free range is large enough
                }
            } else {
                const size_t i = rng() % live.size();
                if (!a.release(live[i].first)) return 4;
                live.erase(live.begin() + i);
            }
            if (!a.check()) return 5;
        }
        for (auto &l : live) a.release(l.first);
        if (a.used() != 0 || a.largest_free() != size || !a.check()) return 6;
        if (a.release(12345)) return 7;  // not a live block
    }
    std::puts("ok");
    return 0;
}
"""


def test_arena_allocator_randomized():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        open(src, "w").write(HARNESS)
        subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1208_0302_gb300", "csrc"),
                        src, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.returncode
        assert r.stdout.strip() == "ok"
