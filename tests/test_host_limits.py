"""Host-side limits the kernels rely on, checked without a GPU: the shear-warp sweep's steps
per launch pair (sw_slices) keep a chunk's voxel indices below 2^24 (the kernels split them
through a float reciprocal) and its ray states within their memory bound.  A small host
program includes the library's internal header and prints the values."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2401_14051_gb300", "csrc")
SIZES = [1, 2, 3, 5, 31, 64, 100, 255, 256, 257, 300, 512, 700, 1000, 1024, 1100, 1448, 1449,
         2048, 2896, 2897, 4000, 4096]

PROGRAM = r"""
#include <cstdio>
#include "nis_internal.h"
int main() {
    const int sizes[] = {%s};
    for (int n : sizes) std::printf("%%d %%d\n", n, nis::sw_slices(n));
    return 0;
}
"""


@pytest.fixture(scope="module")
def slices(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("limits")
    src, exe = d / "limits.cu", d / "limits"
    src.write_text(PROGRAM % ", ".join(map(str, SIZES)))
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {int(a): int(b) for a, b in (line.split() for line in out.split("\n") if line)}


def test_sw_slices_bounds(slices):
    assert sorted(slices) == sorted(SIZES)
    for n, s in slices.items():
        assert 1 <= s <= 32, (n, s)
        # a chunk's voxel launch indexes s slices of n^2 voxels, 0 .. s n^2 - 1: below 2^24
        # up to n = 4096
        assert s * n * n <= 1 << 24, (n, s)
        # ray states of the finest level: (2 n + 3)^2 rays at most, 8 bytes per step kept;
        # above the floor of 2 steps they stay within 256 MiB
        if s > 2:
            assert s * (2 * n + 3) ** 2 * 8 <= 256 * 2 ** 20, (n, s)


def test_sw_slices_of_the_benchmark_grids(slices):
    # 256^3: chunks of 32 steps (16 launches for the sweep); 1024^3: chunks of 7
    assert slices[256] == 32 and slices[1024] == 7
    assert slices[1] == 32 and slices[4096] == 1
