"""Host-side checks of the launch-shape rule of the marching kernels (march_len in
csrc/launch.cuh), compiled into a small host program with nvcc and run on the CPU (no
GPU call).  The rule picks the items per thread K in 8..1 that minimises (waves of
resident 128-thread blocks) x (K + start-up), ties to the larger K; these tests check
it against an exhaustive evaluation of that objective and against the launch shapes
the kernels take on the 512^2 and 256^3 workloads."""
import itertools
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2110_03732_gb300", "csrc")
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"

pytestmark = pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")

CASES = [(n, other, nsm, bps, c0)
         for n, other in [(1, 1), (7, 3), (64, 64), (96, 96), (256, 256), (400, 1), (512, 512), (512, 513),
                          (1024, 1024), (256, 65536), (48, 1760), (4095, 4096)]
         for nsm in (1, 16, 152)
         for bps in (1, 2, 3, 5)
         for c0 in (0.6, 1.0)]


@pytest.fixture(scope="module")
def march_len(tmp_path_factory):
    d = tmp_path_factory.mktemp("launch")
    src = d / "probe.cu"
    lines = ["#include <cstdio>", '#include "launch.cuh"',
             "namespace grmhd { thread_local bool launch_overlap = false; }", "int main() {"]
    for n, other, nsm, bps, c0 in CASES:
        lines.append(f'  std::printf("%d\\n", grmhd::march_len({n}, {other}LL, {nsm}, {bps}, {c0}));')
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = d / "probe"
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split()
    return {case: int(k) for case, k in zip(CASES, out)}


def objective(n, other, nsm, bps, c0, K):
    blocks = ((n + K) // K * other + 127) // 128
    slots = nsm * max(bps, 1)
    return -(-blocks // slots) * (K + c0)


def test_march_len_minimises_the_objective(march_len):
    for case, K in march_len.items():
        assert 1 <= K <= 8, case
        vals = {k: objective(*case, k) for k in range(1, 9)}
        best = min(vals.values())
        assert vals[K] <= best * (1 + 1e-9), (case, K, vals)
        # ties go to the larger K
        assert all(vals[k] > best * (1 + 1e-12) for k in range(K + 1, 9)), (case, K, vals)


def test_march_len_on_the_workloads(march_len):
    # 512^2: 513 faces per line, two FP64 flux blocks per SM -> 7 faces (296 blocks, one
    # wave of 304); with three blocks the rule would take 5
    assert march_len[(512, 512, 152, 2, 0.6)] == 7
    assert march_len[(512, 512, 152, 3, 0.6)] == 5
    # the 512^2 edge EMF along y (5 blocks per SM) marches 3 edges
    assert march_len[(512, 513, 152, 5, 0.6)] == 3
    # small grids take one item per thread for parallelism
    assert march_len[(64, 64, 152, 2, 0.6)] == 1
    # the 256^3 star: many waves, the longest march with the least ragged tail
    assert march_len[(256, 65536, 152, 2, 0.6)] == 7


def test_march_len_small_grids_never_exceed_one_wave_needlessly(march_len):
    # when even K = 1 fits in one wave, K = 1 is chosen (the waves are equal and the
    # march is shortest)
    for (n, other, nsm, bps, c0), K in march_len.items():
        if ((n + 1) * other + 127) // 128 <= nsm * bps:
            assert K == 1, (n, other, nsm, bps, c0, K)
