"""The multiply-high divider of the spectral index decode (fastdiv.h),
compiled for the host with g++, against the hardware division: every
divisor up to 4200 (all grid extents and half-spectrum row lengths) on the
dividends where an off-by-one would show (multiples of d and their
neighbours, powers of two, the top of the 32-bit range), and random
divisor/dividend pairs over the whole 32-bit range."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_2304_01125_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <random>
#include "fastdiv.h"
using fatfft::FastDiv; using fatfft::fdiv; using fatfft::make_fastdiv;
static long bad = 0, n = 0;
static void chk(uint32_t x, const FastDiv& f) {
    ++n;
    if (fdiv(x, f) != x / f.d) { if (bad < 5) std::printf("x=%u d=%u\n", x, f.d); ++bad; }
}
int main() {
    for (uint32_t d = 1; d <= 4200; ++d) {
        const FastDiv f = make_fastdiv(d);
        for (uint32_t x = 0; x < 3 * d + 5; ++x) chk(x, f);
        for (uint64_t q = 1; q * d <= 0xffffffffull; q = q * 3 + 1) {
            const uint32_t x = (uint32_t)(q * d);
            chk(x, f); chk(x - 1, f);
            if (x != 0xffffffffu) chk(x + 1, f);
        }
        for (int b = 0; b < 32; ++b) { chk(1u << b, f); chk((1u << b) - 1, f); }
        chk(0xffffffffu, f); chk(0xfffffffeu, f); chk(0x80000000u, f);
    }
    std::mt19937_64 rng(12345);
    for (int t = 0; t < 2000000; ++t) {
        uint32_t d = (uint32_t)rng();
        if (d == 0) d = 1;
        d >>= (rng() % 32);
        if (d == 0) d = 1;
        const FastDiv f = make_fastdiv(d);
        chk((uint32_t)rng(), f);
        chk((uint32_t)(rng() % 4096) * d, f);
    }
    std::printf("checked %ld, wrong %ld\n", n, bad);
    return bad != 0;
}
"""


def test_fastdiv_matches_hardware_division(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    src = tmp_path / "fd.cpp"
    src.write_text(SRC)
    exe = tmp_path / "fd"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "wrong 0" in res.stdout
