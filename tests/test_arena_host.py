"""The serving loop's first-fit arena (csrc/arena.h) on the CPU: randomized allocate / release
sequences against a brute-force model of the region.  Every allocation must lie in free space,
be the lowest-offset free run that fits (first fit), fail only when no free run fits, and after
every step the arena's free list must equal the maximal free runs of the model (coalescing)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_00628_gb300", "csrc")

DRIVER = r"""
#include "arena.h"
#include <cstdio>
#include <random>
#include <utility>
#include <vector>
using swk::Arena;

// maximal runs of free units of the model, in offset order
static std::vector<std::pair<size_t, size_t>> runs(const std::vector<char>& used) {
    std::vector<std::pair<size_t, size_t>> r;
    for (size_t i = 0; i < used.size();) {
        if (used[i]) { ++i; continue; }
        size_t j = i;
        while (j < used.size() && !used[j]) ++j;
        r.push_back({i, j - i});
        i = j;
    }
    return r;
}

int main() {
    std::mt19937_64 rng(20231);
    for (int trial = 0; trial < 300; ++trial) {
        const size_t N = 1 + rng() % 2048;
        Arena a;
        a.init(N);
        std::vector<char> used(N, 0);
        std::vector<std::pair<size_t, size_t>> live;
        for (int step = 0; step < 300; ++step) {
            if (live.empty() || rng() % 3 != 0) {
                const size_t n = rng() % 200;
                size_t off = 12345;
                const bool ok = a.alloc(n, &off);
                if (n == 0) {
                    if (!ok || off != 0) { std::printf("zero-size alloc\n"); return 1; }
                    continue;
                }
                size_t want = (size_t)-1;
                for (const auto& r : runs(used))
                    if (r.second >= n) { want = r.first; break; }
                if (ok != (want != (size_t)-1) || (ok && off != want)) {
                    std::printf("first fit: trial %d step %d n %zu ok %d off %zu want %zu\n", trial, step, n,
                                (int)ok, off, want);
                    return 1;
                }
                if (ok) {
                    for (size_t i = off; i < off + n; ++i) used[i] = 1;
                    live.push_back({off, n});
                }
            } else {
                const size_t k = rng() % live.size();
                a.release(live[k].first, live[k].second);
                for (size_t i = live[k].first; i < live[k].first + live[k].second; ++i) used[i] = 0;
                live.erase(live.begin() + (long)k);
            }
            const auto r = runs(used);
            if (r.size() != a.free_.size()) { std::printf("free list size: trial %d step %d\n", trial, step); return 1; }
            size_t idx = 0;
            for (const auto& f : a.free_) {
                if (f.first != r[idx].first || f.second != r[idx].second) {
                    std::printf("free run mismatch: trial %d step %d\n", trial, step);
                    return 1;
                }
                ++idx;
            }
        }
        for (const auto& l : live) a.release(l.first, l.second);
        if (a.free_.size() != 1 || a.free_.begin()->first != 0 || a.free_.begin()->second != N) {
            std::printf("not whole after releasing everything: trial %d\n", trial);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
"""


def test_arena_first_fit_and_coalescing(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    src = tmp_path / "arena_driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "arena_driver"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
