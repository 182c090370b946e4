"""The store's keyframe-id map (tmap::IdMap, host code of the library) against
std::unordered_map under random inserts, lookups and erases, compiled with nvcc as host code
and run on the CPU (no device calls)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <random>
#include <unordered_map>
#include "runtime.h"
int main() {
    tmap::IdMap m;
    std::unordered_map<uint64_t, int> ref;
    std::mt19937_64 rng(7);
    for (int it = 0; it < 200000; ++it) {
        const uint64_t k = rng() % 3000 + ((it % 7 == 0) ? (1ull << 40) : 0);  // dense and far ids
        const int op = (int)(rng() % 4);
        if (op == 0 || op == 1) {
            const int v = (int)(rng() % 100000);
            m[k] = v;
            ref[k] = v;
        } else if (op == 2) {
            if (m.erase(k) != ref.erase(k)) { printf("erase mismatch\n"); return 1; }
        } else {
            auto a = m.find(k);
            auto b = ref.find(k);
            if ((a == m.end()) != (b == ref.end())) { printf("find mismatch\n"); return 1; }
            if (a != m.end() && (a->second != b->second || a->first != k)) { printf("value mismatch\n"); return 1; }
        }
        if (m.size() != ref.size()) { printf("size mismatch\n"); return 1; }
    }
    for (const auto &kv : ref)
        if (!m.count(kv.first) || m.find(kv.first)->second != kv.second) { printf("final mismatch\n"); return 1; }
    auto it = m.find(ref.begin()->first);
    m.erase(it);
    if (m.count(ref.begin()->first)) { printf("erase by iterator\n"); return 1; }
    printf("ok %zu\n", m.size());
    return 0;
}
'''


def test_idmap_matches_unordered_map():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = os.path.join(ROOT, "tests", "_build", "idmap_%d" % os.getpid())
    os.makedirs(d, exist_ok=True)
    try:
        src = os.path.join(d, "idmap.cu")
        open(src, "w").write(SRC)
        exe = os.path.join(d, "idmap")
        subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_2511_02036_gb300", "csrc"), src, "-o", exe],
                       check=True, capture_output=True, text=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    finally:
        shutil.rmtree(d, ignore_errors=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
