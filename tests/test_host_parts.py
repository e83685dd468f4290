"""The library's host worker pool (csrc/host_parts.h: run_parts over a
persistent set of threads, and the allocator that leaves new elements unset),
compiled on its own with the host C++ compiler: every part of every job runs
exactly once, also with concurrent callers, nested calls from inside a part,
and a part that throws on the calling thread."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1401_1757_gb300", "csrc")

SRC = r"""
#include "host_parts.h"
#include <cstdio>
#include <stdexcept>
#include <thread>
#include <vector>

static bool check(std::vector<std::atomic<int>>& hits, int want) {
    for (auto& h : hits)
        if (h.load() != want) return false;
    return true;
}

int main() {
    using rsv::run_parts;
    // many jobs of different widths, each part exactly once
    for (int rep = 0; rep < 3000; ++rep) {
        const int T = 1 + rep % 19;
        std::vector<std::atomic<int>> hits(T);
        run_parts(T, [&](int k) { hits[k]++; });
        if (!check(hits, 1)) { std::printf("FAIL widths %d\n", T); return 1; }
    }
    // two callers at once: the one that finds the pool busy starts its own threads
    bool ok[2] = {true, true};
    std::vector<std::thread> callers;
    for (int c = 0; c < 2; ++c)
        callers.emplace_back([&, c] {
            for (int rep = 0; rep < 1000; ++rep) {
                std::vector<std::atomic<int>> hits(16);
                run_parts(16, [&](int k) { hits[k]++; });
                if (!check(hits, 1)) ok[c] = false;
            }
        });
    for (auto& t : callers) t.join();
    if (!ok[0] || !ok[1]) { std::printf("FAIL concurrent\n"); return 1; }
    // a part that splits its own work again
    std::vector<std::atomic<int>> inner(8 * 4);
    run_parts(8, [&](int k) { run_parts(4, [&](int j) { inner[4 * k + j]++; }); });
    if (!check(inner, 1)) { std::printf("FAIL nested\n"); return 1; }
    // an exception from a part run by the caller reaches it after every part ran
    std::vector<std::atomic<int>> hits(1);
    try {
        run_parts(1, [&](int k) { hits[k]++; throw std::runtime_error("part"); });
        std::printf("FAIL no exception\n");
        return 1;
    } catch (const std::runtime_error&) {
    }
    if (!check(hits, 1)) { std::printf("FAIL exception\n"); return 1; }
    // the allocator: resize keeps values written before, new elements are writable
    std::vector<int, rsv::DefaultInit<int>> v(4, 7);
    v.resize(1 << 20);
    v[(1 << 20) - 1] = 3;
    if (v[0] != 7 || v[3] != 7 || v[(1 << 20) - 1] != 3) { std::printf("FAIL allocator\n"); return 1; }
    std::printf("OK\n");
    return 0;
}
"""


def test_run_parts_pool(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "pool.cpp"
    src.write_text(SRC)
    exe = tmp_path / "pool"
    subprocess.run([cxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr
