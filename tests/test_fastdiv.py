"""The invariant-divisor division used for grid coordinates (host path of the
library's own header, compiled with nvcc for the CPU) equals integer division
on edge cases and random dividends (Granlund-Montgomery round-up method)."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cstdint>
#include <random>
#include "tsz_common.cuh"
int main() {
    std::mt19937_64 r(7);
    long bad = 0;
    const uint32_t ds[] = {1u, 2u, 3u, 7u, 31u, 32u, 33u, 100u, 128u, 129u, 384u, 512u, 1800u, 3600u, 4096u,
                           65537u, 1u << 20, (1u << 31) - 1u, 1u << 31, 0xFFFFFFFFu};
    for (uint32_t d : ds) {
        tsz::FastDiv f = tsz::make_fastdiv(d);
        const uint32_t edge[] = {0u, 1u, d - 1u, d, d + 1u, 2u * d, 0x7FFFFFFFu, 0x80000000u, 0xFFFFFFFFu};
        for (uint32_t n : edge) bad += tsz::fdiv(n, f) != n / d;
        for (int k = 0; k < 100000; k++) { uint32_t n = (uint32_t)r(); bad += tsz::fdiv(n, f) != n / d; }
    }
    for (int k = 0; k < 5000; k++) {
        uint32_t d = (uint32_t)(r() % 0x7FFFFFFFu) + 1u;
        tsz::FastDiv f = tsz::make_fastdiv(d);
        for (int j = 0; j < 50; j++) { uint32_t n = (uint32_t)r(); bad += tsz::fdiv(n, f) != n / d; }
    }
    printf("%ld\n", bad);
    return bad != 0;
}
'''


def test_fastdiv_exact():
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "fd.cu")
        exe = os.path.join(d, "fd")
        open(src, "w").write(SRC)
        subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I",
                               os.path.join(ROOT, "paper_2602_17552_gb300", "csrc"), src, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0 and out.stdout.strip() == "0", out.stdout + out.stderr
