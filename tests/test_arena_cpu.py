"""The serving arena's sub-allocator (csrc/ci_arena.h, host-only C++) against
a granule-by-granule model, compiled with g++ on the CPU: after every one of
tens of thousands of random allocations (first fit from the bottom, highest fit
from the top) and releases, the free list equals the model's maximal free runs
(so neighbours always coalesce), each allocation is the lowest (or highest)
fitting place, a refused allocation had no fitting gap, and the used and peak
byte counts match; releasing everything leaves one block of the whole arena."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1112_5239_gb300", "csrc")

DRIVER = r'''
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include "ci_arena.h"

struct Block { uint64_t off, bytes; };

static int fail(const char *what, long step) { std::printf("FAIL %s at step %ld\n", what, step); return 1; }

int main(int argc, char **argv) {
    const uint64_t G = 256, n_gran = std::strtoull(argv[1], nullptr, 10);
    const long steps = std::atol(argv[2]);
    std::mt19937_64 rng(std::strtoull(argv[3], nullptr, 10));
    ci::Arena a;
    a.init(n_gran * G);
    std::vector<char> busy(n_gran, 0);
    std::vector<Block> live;
    uint64_t used = 0, peak = 0;
    for (long step = 0; step < steps; ++step) {
        const int op = (int)(rng() % 10);
        if (op < 6 || live.empty()) {
            const bool high = (rng() & 1) != 0;
            const uint64_t bytes = 1 + rng() % (G * (1 + rng() % 64));  // 1 B .. 64 granules
            const uint64_t g = (bytes + G - 1) / G;
            // model: the fitting runs, lowest and highest
            long lo = -1, hi = -1;
            for (uint64_t i = 0; i < n_gran;) {
                if (busy[i]) { ++i; continue; }
                uint64_t j = i;
                while (j < n_gran && !busy[j]) ++j;
                if (j - i >= g) { if (lo < 0) lo = (long)i; hi = (long)(j - g); }
                i = j;
            }
            uint64_t off = 0;
            const bool ok = high ? a.alloc_high(bytes, &off) : a.alloc(bytes, &off);
            if (!ok) { if (lo >= 0) return fail("refused although a gap fits", step); continue; }
            if (lo < 0) return fail("granted without a fitting gap", step);
            if (off % G) return fail("unaligned offset", step);
            const uint64_t want = (uint64_t)(high ? hi : lo) * G;
            if (off != want) return fail(high ? "not the highest fit" : "not the lowest fit", step);
            for (uint64_t i = off / G; i < off / G + g; ++i) {
                if (busy[i]) return fail("overlap", step);
                busy[i] = 1;
            }
            live.push_back({off, bytes});
            used += g * G;
            peak = used > peak ? used : peak;
        } else {
            const size_t k = rng() % live.size();
            const Block b = live[k];
            live[k] = live.back();
            live.pop_back();
            a.release(b.off, b.bytes);
            const uint64_t g = (b.bytes + G - 1) / G;
            for (uint64_t i = b.off / G; i < b.off / G + g; ++i) busy[i] = 0;
            used -= g * G;
        }
        if (a.used() != used || a.peak() != peak) return fail("used / peak accounting", step);
        // the free list is exactly the model's maximal free runs, in address order
        std::vector<Block> runs, list;
        for (uint64_t i = 0; i < n_gran;) {
            if (busy[i]) { ++i; continue; }
            uint64_t j = i;
            while (j < n_gran && !busy[j]) ++j;
            runs.push_back({i * G, (j - i) * G});
            i = j;
        }
        a.for_each_free([&](uint64_t o, uint64_t b) { list.push_back({o, b}); });
        if (runs.size() != list.size()) return fail("free list is not the maximal runs (count)", step);
        for (size_t i = 0; i < runs.size(); ++i)
            if (runs[i].off != list[i].off || runs[i].bytes != list[i].bytes)
                return fail("free list is not the maximal runs", step);
    }
    // release everything: one block of the whole arena again
    for (const Block &b : live) a.release(b.off, b.bytes);
    uint64_t off = 0;
    if (a.used() != 0 || !a.alloc(n_gran * G, &off) || off != 0) return fail("full arena after releases", steps);
    std::printf("ok\n");
    return 0;
}
'''


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
@pytest.mark.parametrize("n_gran,steps,seed", [(64, 20000, 1), (1024, 20000, 2), (4096, 5000, 3)])
def test_arena_against_granule_model(tmp_path, n_gran, steps, seed):
    src, exe = tmp_path / "arena_driver.cpp", tmp_path / "arena_driver"
    src.write_text(DRIVER)
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)])
    r = subprocess.run([str(exe), str(n_gran), str(steps), str(seed)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
