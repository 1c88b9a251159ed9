"""The polarized tracers' parallel transport of the reference covector (csrc/synch.cuh
transport_rhs: df_mu/dlambda = Gamma^alpha_{mu beta} k^beta f_alpha in closed form), built for the
host from the same source, against the oracle's (Christoffel symbols from complex-step metric
derivatives): 2000 random states at 1.5 to 1000 M, spins of both signs."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_07417_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector_types.h>
#include "synch.cuh"
int main()
{
    double a, v[11];
    while (std::scanf("%lf %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf", &a, v, v + 1, v + 2, v + 3,
                      v + 4, v + 5, v + 6, v + 7, v + 8, v + 9, v + 10) == 12) {
        art::RayState<double> s{v[0], v[1], v[2], v[3], v[4], v[5]};
        double df[4];
        art::transport_rhs<double>(s, v[6], v + 7, a, a * a, df);
        std::printf("%.17g %.17g %.17g %.17g\n", df[0], df[1], df[2], df[3]);
    }
    return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    return None


def test_transport_rhs_matches_oracle(tmp_path):
    gxx, inc = shutil.which("g++"), _cuda_include()
    if gxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    src = tmp_path / "tr.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "tr"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                   check=True)
    rng = np.random.default_rng(9)
    rows = []
    for _ in range(2000):
        a = rng.uniform(-0.99, 0.99)
        rad = 10 ** rng.uniform(np.log10(1.5), 3.0)
        d = rng.normal(size=3)
        x = rad * d / np.linalg.norm(d)
        k = rng.normal(size=3)
        kt = -rng.uniform(0.5, 2.0)
        f = rng.normal(size=4)
        rows.append((a, *x, *k, kt, *f))
    inp = "\n".join(" ".join(f"{v:.17g}" for v in r) for r in rows) + "\n"
    out = subprocess.run([str(exe)], input=inp, check=True, capture_output=True, text=True).stdout
    got = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    worst = 0.0
    for row, g in zip(rows, got):
        a, x0, y0, z0, kx, ky, kz, kt, f0, f1, f2, f3 = row
        job = O.make_job(**W.kerr_disk_2049(a=a, n0x=3, n0y=3, levels=0))
        y12 = np.array([0.0, x0, y0, z0, kt, kx, ky, kz, f0, f1, f2, f3])
        want = O.transport_rhs(job, y12)
        worst = max(worst, np.abs(g - want).max() / max(np.abs(want).max(), 1e-300))
    assert worst < 1e-8, worst
