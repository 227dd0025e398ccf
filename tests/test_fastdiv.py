"""Division by a launch-invariant divisor as a multiply-high and two shifts (Granlund and
Montgomery, PLDI 1994, Fig. 4.1), used by the evaluation kernels for the unit and span
indices: the constants come from the library's own host code (compiled here with g++
from the internal header) and the device arithmetic, restated with 64-bit integers, must
equal floor(n / d) for every divisor tried and every n tried, up to 2^32 - 1."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROGRAM = r'''
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include "paper_2503_14160_gb300/csrc/cp_internal.cuh"
int main(int argc, char **argv) {
    for (int i = 1; i < argc; ++i) {
        const cp::FastDiv f = cp::fast_div((uint32_t)strtoul(argv[i], nullptr, 10));
        printf("%u %u %u\n", f.m, f.sh1, f.sh2);
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def constants(tmp_path_factory):
    gxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("fastdiv")
    src, exe = d / "fd.cpp", d / "fd"
    src.write_text(PROGRAM)
    subprocess.run([gxx, "-std=c++17", "-I", ROOT, "-I", inc, str(src), "-o", str(exe)], check=True)

    def get(divisors):
        out = subprocess.run([str(exe)] + [str(int(x)) for x in divisors], check=True,
                             capture_output=True, text=True).stdout.split()
        return np.array(out, dtype=np.uint64).reshape(-1, 3)
    return get


def _fdiv(n, m, sh1, sh2):
    t = (m * n) >> np.uint64(32)
    return (t + ((n - t) >> sh1)) >> sh2


def test_exact_for_every_small_divisor_and_edge_numerators(constants):
    divisors = np.arange(1, 4097, dtype=np.uint64)
    c = constants(divisors)
    rng = np.random.default_rng(0)
    base = np.concatenate([np.arange(0, 5000), rng.integers(0, 2 ** 32, 2000),
                           [2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1]]).astype(np.uint64)
    for d, (m, s1, s2) in zip(divisors, c):
        k = rng.integers(0, (2 ** 32 - 2) // int(d), 200).astype(np.uint64)
        n = np.concatenate([base, k * d, k * d + d - np.uint64(1)])
        np.testing.assert_array_equal(_fdiv(n, m, s1, s2), n // d)


def test_exact_for_large_divisors(constants):
    rng = np.random.default_rng(1)
    divisors = np.concatenate([rng.integers(4097, 2 ** 32, 300),
                               [2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, 2 ** 32 - 1]]).astype(np.uint64)
    c = constants(divisors)
    n = np.concatenate([rng.integers(0, 2 ** 32, 20000), [0, 1, 2 ** 32 - 1]]).astype(np.uint64)
    for d, (m, s1, s2) in zip(divisors, c):
        nn = np.concatenate([n, [d - np.uint64(1), d, (np.uint64(2 ** 32 - 1) // d) * d]]).astype(np.uint64)
        np.testing.assert_array_equal(_fdiv(nn, m, s1, s2), nn // d)
