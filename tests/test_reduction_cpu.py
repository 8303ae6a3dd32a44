"""Host-side sizing of the two-level grid reduction (no GPU): the group
size, the group count and the partials/ticket capacities the library
allocates, compiled from the library's own header with nvcc (host code)
and checked for every block count up to 2^17 and batch sizes 1..64.

The device code relies on: at most as many groups as blocks per group (the
ticket array holds 1 + G entries), one group for every single-value launch
up to 2048 blocks, and the capacity bound quantities * (blocks + G) holding
for every smaller grid too (a lattice sizes its scratch once, for its
largest launch)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1411_5219_gb300", "csrc")

PROGRAM = r"""
#include "qcd_internal.cuh"
#include <cstdio>
using namespace qcd;
int main()
{
    long bad = 0;
    for (unsigned P : {1u, 2u, 4u, 16u, 32u, 64u}) {
        unsigned prev_g = 0;
        size_t worst_ratio_num = 0;
        for (unsigned nb = 1; nb <= (1u << 17); ++nb) {
            const unsigned G = red_group_size(nb, P), ng = (nb + G - 1) / G;
            if (ng > G) ++bad;                              // tickets: 1 + G suffice
            if (G < prev_g) ++bad;                          // G does not shrink with more blocks
            if ((G & (G - 1)) != 0 || G < 64 || G * P < 2048) ++bad;
            if (P == 1 && nb <= 2048 && ng != 1) ++bad;     // one level for small single-value grids
            if ((size_t)P * (nb + ng) > red_partials_needed(P, nb)) ++bad;
            prev_g = G;
        }
        // a capacity sized for B blocks holds every grid of nb <= B blocks
        for (unsigned B : {1u, 63u, 864u, 2048u, 4097u, 16384u, 100000u})
            for (unsigned nb = 1; nb <= B; nb += (B > 5000 ? 7 : 1)) {
                const unsigned G = red_group_size(nb, P), ng = (nb + G - 1) / G;
                if ((size_t)P * (nb + ng) > red_partials_needed(P, B)) ++bad;
            }
    }
    printf("%ld\n", bad);
    return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_reduction_group_sizing(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "red.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "red"
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out == ["0"], out
