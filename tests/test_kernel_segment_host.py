"""The polarized tracers' constant-coefficient Stokes segment (csrc/synch.cuh segment_pol: the
closed-form exponential of the Mueller matrix with the attenuation folded into the hyperbolic
functions), built for the host from the same source, against the oracle's (the exponential of the
augmented 5 x 5 matrix by scaling and squaring): propagator and source of one segment from the
identity, over optically thin to thick segments, weak to strong Faraday terms and the degenerate
cases (no polarized coefficients, pure rotation, pure dichroism)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_07417_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector_types.h>
#include "synch.cuh"
int main()
{
    double K[7], J[4], h;
    while (std::scanf("%lf %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf", K, K + 1, K + 2, K + 3,
                      K + 4, K + 5, K + 6, J, J + 1, J + 2, J + 3, &h) == 12) {
        double P[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1}, acc[4] = {0, 0, 0, 0};
        art::segment_pol<double>(K, J, h, P, acc);
        for (int i = 0; i < 16; ++i) std::printf("%.17g ", P[i]);
        std::printf("%.17g %.17g %.17g %.17g\n", acc[0], acc[1], acc[2], acc[3]);
    }
    return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    return None


def _cases(rng):
    out = []
    for _ in range(1500):
        pol = rng.normal(size=3) * 10 ** rng.uniform(-3, 0)
        aI = np.linalg.norm(pol) * (1 + rng.uniform(0, 2))      # physical: aI >= |(aQ, aU, aV)|
        rot = rng.normal(size=3) * 10 ** rng.uniform(-3, 1.5)
        J = np.concatenate([[abs(rng.normal())], rng.normal(size=3) * 0.3])
        h = 10 ** rng.uniform(-2, 1.5)
        out.append((aI, *pol, *rot, *J, h))
    out.append((0.5, 0, 0, 0, 0, 0, 0, 1.0, 0, 0, 0, 1.0))           # unpolarized slab
    out.append((0.0, 0, 0, 0, 2.0, 0.5, 1.0, 0.0, 0.3, 0.2, 0.1, 0.7))  # pure rotation, no emission
    out.append((0.4, 0.3, 0.1, 0.0, 0, 0, 0, 0.2, 0.1, 0, 0, 2.0))     # pure dichroism
    return out


def test_segment_matches_oracle(tmp_path):
    gxx, inc = shutil.which("g++"), _cuda_include()
    if gxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    src = tmp_path / "seg.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "seg"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                   check=True)
    rows = _cases(np.random.default_rng(3))
    inp = "\n".join(" ".join(f"{v:.17g}" for v in r) for r in rows) + "\n"
    out = subprocess.run([str(exe)], input=inp, check=True, capture_output=True, text=True).stdout
    got = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    worst_E = worst_X = 0.0
    for row, g in zip(rows, got):
        K7, J4, h = np.array(row[:7]), np.array(row[7:11]), row[11]
        E, X = O.segment(K7, J4, h)
        E = np.asarray(E).reshape(16)
        worst_E = max(worst_E, np.abs(g[:16] - E).max() / max(np.abs(E).max(), 1e-300))
        worst_X = max(worst_X, np.abs(g[16:] - X).max() / max(np.abs(X).max(), 1e-300))
    assert worst_E < 1e-9 and worst_X < 1e-9, (worst_E, worst_X)
