"""The tracer's modified Bessel functions K_0, K_1, K_2 of 1/Theta_e (csrc/synch.cuh bessel_k012:
the polynomial fits of Abramowitz & Stegun 9.8.1-9.8.8, unscaled for x <= 2 and scaled by e^x
above, with the flag telling which), built for the host from the same source, against the
oracle's K_n from their integral representation K_n(x) = int_0^inf e^{-x cosh t} cosh(n t) dt."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_07417_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <vector_types.h>
#include "synch.cuh"
int main()
{
    double x;
    while (std::scanf("%lf", &x) == 1) {
        double K0, K1, K2;
        const bool scaled = art::bessel_k012<double>(x, 1.0 / x, std::log(x), K0, K1, K2);
        std::printf("%d %.17g %.17g %.17g\n", scaled ? 1 : 0, K0, K1, K2);
    }
    return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    return None


def test_bessel_fits_match_the_integral(tmp_path):
    gxx, inc = shutil.which("g++"), _cuda_include()
    if gxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    src = tmp_path / "bk.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "bk"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                   check=True)
    xs = np.concatenate([np.geomspace(1e-3, 50.0, 200), [2.0, np.nextafter(2.0, 3.0), 1.0]])
    out = subprocess.run([str(exe)], input="\n".join(f"{x:.17g}" for x in xs) + "\n",
                         check=True, capture_output=True, text=True).stdout.split("\n")
    for x, line in zip(xs, out):
        sc, *K = line.split()
        assert int(sc) == (1 if x > 2.0 else 0), x
        scale = np.exp(x) if x > 2.0 else 1.0
        for n in range(3):
            want = O.bessel_k(n, x) * scale
            assert float(K[n]) == pytest.approx(want, rel=2e-6), (n, x)
