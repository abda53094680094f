"""The predictor sum on the integer pipe (wsum_int, lb_device.cuh, used by the
grid and one-CTA sweeps), compiled for the host from the kernel source and
checked on the CPU.

The first iterate of a step extrapolates the last n corrections with the
weights (-1)^(k+1) C(n, k) (polynomial extrapolation through equally spaced
points, Appendix A's implicit-midpoint inner solve started from a predicted
iterate).  The sum is computed exactly in 64-bit integers after aligning the
significands; these tests pin it to exact rational arithmetic, to the
extrapolation's defining property (a polynomial of degree < n is continued
exactly) and to its handling of non-finite and extreme inputs."""

import importlib
import os
import shutil
import struct
import subprocess
from fractions import Fraction
from math import comb

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "wsum_harness.cu")


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dbl(u: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def _weights(n: int):
    """Weight of x_i (i = 0 the oldest of n entries): (-1)^(k+1) C(n, k), k = n - i."""
    return [(1 if (n - i) % 2 else -1) * comb(n, n - i) for i in range(n)]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    B = importlib.import_module("paper_2110_10310_gb300.build")

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("wsum") / "wsum")
    # the kernels are carried as PTX only (nothing runs on a device here),
    # which spares the device assembler's time
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=compute_103a", "-O2",
           "--expt-relaxed-constexpr", "-I", B.INCLUDE, "-I", B.CSRC, "-o", exe, HARNESS]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def _run(exe, cases):
    inp = "".join(f"{len(c)} " + " ".join(f"{_bits(float(x)):016x}" for x in c) + "\n" for c in cases)
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return [_dbl(int(t, 16)) for t in r.stdout.split()]


def test_sum_is_the_weighted_sum_within_its_bound(harness):
    """Against the exact rational sum: the error stays below
    2 sum|w| 2^-52 max|x| (aligned-term and final truncation), plus the
    flush of results below the normal range."""
    rng = np.random.default_rng(2110)
    cases = []
    for n in (8, 9, 10):
        for t in range(400):
            kind = t % 4
            if kind == 0:
                x = rng.uniform(-1, 1, n)
            elif kind == 1:  # exponents spread over 2^-60 .. 2^10
                x = rng.uniform(-1, 1, n) * np.exp2(rng.integers(-60, 11, n).astype(float))
            elif kind == 2:  # a smooth sequence: the sum cancels to far below the entries
                i = np.arange(n, dtype=float)
                x = (1e-3 * (1 + i) + 2e-5 * i**2 - 3e-7 * i**3) * (1 + 1e-9 * rng.uniform(-1, 1, n))
            else:  # subnormal and zero entries
                x = rng.uniform(-1, 1, n) * np.exp2(rng.integers(-1070, -1030, n).astype(float))
                x[rng.integers(0, n)] = 0.0
            cases.append(list(x))
    got = _run(harness, cases)
    for c, r in zip(cases, got):
        n = len(c)
        w = _weights(n)
        exact = sum(Fraction(wi) * Fraction(xi) for wi, xi in zip(w, c))
        mx = max(abs(Fraction(xi)) for xi in c)
        bound = 2 * sum(abs(wi) for wi in w) * mx / 2**52 + Fraction(1, 2**1021)
        assert abs(Fraction(r) - exact) <= bound, (c, r, float(exact))


@pytest.mark.parametrize("n", [8, 9, 10])
def test_polynomials_of_lower_degree_are_continued_exactly(harness, n):
    """x_i = p(i) for i = 1..n with deg p < n: the sum is p(n + 1), exactly
    (integer values, so every step of the integer sum is exact).  Pins the
    weights, their signs and the ring order (x_0 the oldest)."""
    rng = np.random.default_rng(n)
    cases, want = [], []
    for deg in range(n):
        coef = [int(c) for c in rng.integers(-20, 21, deg + 1)]

        def p(t):
            return sum(c * t**k for k, c in enumerate(coef))

        cases.append([float(p(i)) for i in range(1, n + 1)])
        want.append(float(p(n + 1)))
    assert _run(harness, cases) == want


def test_non_finite_and_extreme_inputs(harness):
    nan, inf = float("nan"), float("inf")
    cases = [
        [1.0, 2.0, nan, 4.0, 5.0, 6.0, 7.0, 8.0, 9.0],
        [1.0, 2.0, inf, 4.0, 5.0, 6.0, 7.0, 8.0, 9.0],
        [(-1.0) ** i * 1.7e308 for i in range(9)],
        [0.0] * 9,
        [-0.0] * 9,
        [5e-324] * 8 + [0.0],
    ]
    r = _run(harness, cases)
    assert np.isnan(r[0]) and np.isnan(r[1])  # a non-finite entry gives NaN
    assert np.isinf(r[2])  # beyond the double range: infinity
    assert r[3] == 0.0 and r[4] == 0.0
    # eight smallest subnormals and a zero: the exact sum, -8 x 2^-1074, lies
    # below the normal range and is flushed to (signed) zero
    assert r[5] == 0.0
