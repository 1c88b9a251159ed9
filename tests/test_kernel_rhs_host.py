"""The tracer's hand-derived Hamilton equations (csrc/kerr.cuh geodesic_rhs, the code every trace
kernel inlines), built for the host from the same source, against the derivatives of the
Kerr-Schild Hamiltonian H = 1/2 (eta^{mu nu} k_mu k_nu - f (l.k)^2) taken here by complex steps:
dx_i/dlambda = dH/dk_i and dk_i/dlambda = -dH/dx_i, and the radius r it returns.  Random states at
1.5 to 1000 M, spins of both signs; FP64 throughout."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_07417_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "kerr.cuh"
int main()
{
    double a, v[7];
    while (std::scanf("%lf %lf %lf %lf %lf %lf %lf %lf", &a, v, v + 1, v + 2, v + 3, v + 4, v + 5,
                      v + 6) == 8) {
        art::RayState<double> s{v[0], v[1], v[2], v[3], v[4], v[5]}, d;
        double ks[5];
        const double r = art::geodesic_rhs<double>(s, v[6], a, a * a, d, ks);
        std::printf("%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", r,
                    d.x, d.y, d.z, d.kx, d.ky, d.kz, ks[0], ks[1], ks[2], ks[3], ks[4]);
    }
    return 0;
}
"""


def _hamiltonian(a, x, k, kt):
    """H of the outgoing Kerr-Schild metric (complex-safe: complex steps go through every term)."""
    X, Y, Z = x
    b = X * X + Y * Y + Z * Z - a * a
    r2 = 0.5 * (b + np.sqrt(b * b + 4 * a * a * Z * Z))
    r = np.sqrt(r2)
    f = 2 * r2 * r / (r2 * r2 + a * a * Z * Z)
    L = ((r * X - a * Y) / (r2 + a * a), (r * Y + a * X) / (r2 + a * a), Z / r)
    lk = -kt - (L[0] * k[0] + L[1] * k[1] + L[2] * k[2])
    return 0.5 * (-kt * kt + k[0] ** 2 + k[1] ** 2 + k[2] ** 2 - f * lk * lk), r, f, L


def test_geodesic_rhs_matches_the_hamiltonian(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "rhs.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "rhs"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    rng = np.random.default_rng(5)
    rows = []
    while len(rows) < 3000:
        a = rng.uniform(-0.99, 0.99)
        rad = 10 ** rng.uniform(np.log10(1.5), 3.0)
        dirn = rng.normal(size=3)
        x = rad * dirn / np.linalg.norm(dirn)
        k = rng.normal(size=3)
        kt = -rng.uniform(0.5, 2.0)
        rows.append((a, *x, *k, kt))
    inp = "\n".join(" ".join(f"{v:.17g}" for v in r) for r in rows) + "\n"
    out = subprocess.run([str(exe)], input=inp, check=True, capture_output=True, text=True).stdout
    got = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    assert got.shape == (len(rows), 12)
    h = 1e-30
    worst = 0.0
    for (a, x0, y0, z0, kx, ky, kz, kt), g in zip(rows, got):
        x = np.array([x0, y0, z0])
        k = np.array([kx, ky, kz])
        _, r, f, L = _hamiltonian(a, x, k, kt)
        dH_dk = np.array([_hamiltonian(a, x, k + 1j * h * e, kt)[0].imag / h for e in np.eye(3)])
        dH_dx = np.array([_hamiltonian(a, x + 1j * h * e, k, kt)[0].imag / h for e in np.eye(3)])
        want = np.concatenate([dH_dk, -dH_dx])
        scale = np.abs(want).max()
        worst = max(worst, np.abs(g[1:7] - want).max() / scale)
        assert g[0] == pytest.approx(r, rel=1e-13)
        assert np.allclose(g[7:], [1 / r, f, *L], rtol=1e-12, atol=0.0)
    assert worst < 1e-9, worst
