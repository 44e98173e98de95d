"""Host check of the multiply-high division (FastDiv / fdiv in csrc/grmhd_device.cuh)
that turns an interior cell index into (i, j, k) in the implicit kernel: compiled with
nvcc into a small host program and run on the CPU (no GPU call).  Every divisor up to
70000 and a spread of larger ones is checked against plain unsigned division on
dividends at and around multiples of the divisor, near 2^32 and at random."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2110_03732_gb300", "csrc")
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"

pytestmark = pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")

PROG = r'''
#include <cstdio>
#include <cstdint>
#include "grmhd_device.cuh"
static uint64_t rng = 88172645463325252ull;
static unsigned next() { rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17; return (unsigned)(rng >> 11); }
int main() {
    unsigned long long checked = 0, bad = 0;
    auto check = [&](unsigned d, unsigned t) {
        const grmhd::FastDiv f = grmhd::make_fastdiv(d);
        checked++;
        if (grmhd::fdiv(t, f) != t / d) { if (bad < 10) std::printf("BAD %u %u\n", d, t); bad++; }
    };
    for (unsigned d = 1; d <= 70000u; d++) {
        const unsigned ts[] = {0u, 1u, d - 1u, d, d + 1u, 2u * d - 1u, 0xffffffffu, 0xfffffffeu, 0x80000000u,
                               0x7fffffffu, (0xffffffffu / d) * d, (0xffffffffu / d) * d - 1u};
        for (unsigned t : ts) check(d, t);
        for (int r = 0; r < 16; r++) check(d, next());
    }
    for (int r = 0; r < 200000; r++) {
        unsigned d = next() >> (next() % 31);
        if (d == 0) d = 1;
        unsigned t = next();
        check(d, t);
        check(d, (t / d) * d);
        check(d, (t / d) * d + d - 1u > (t / d) * d ? (t / d) * d + d - 1u : t);
    }
    for (unsigned k = 0; k < 32; k++) {
        const unsigned d = 1u << k;
        check(d, 0xffffffffu); check(d, d); check(d, d - 1u);
        if (d > 1) { check(d + 1u, 0xffffffffu); check(d - 1u, 0xffffffffu); }
    }
    std::printf("%llu %llu\n", checked, bad);
    return 0;
}
'''


def test_fastdiv_matches_plain_division(tmp_path):
    src = tmp_path / "fastdiv.cu"
    src.write_text(PROG)
    exe = tmp_path / "fastdiv"
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split()
    checked, bad = int(out[-2]), int(out[-1])
    assert checked > 2_000_000 and bad == 0, out[:20]
