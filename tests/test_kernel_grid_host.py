"""The FP64 tracer's fluid-grid emission (csrc/grid.cuh: the integer widening of cell values,
the trilinear lookup in (ln r, theta, phi), u^t, b^mu, the two-temperature plasma and the
thermal-synchrotron coefficients with the table logarithm), built for the host from the same
source, against the oracle's grid model at the RK4 points of oracle rays through the seeded torus;
and the widening against the conversion for every one of the 2^32 floats."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_07417_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(ROOT, "paper_2103_07417_gb300", "lib")

WIDEN = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector_types.h>
#include "grid.cuh"
int main()
{
    unsigned long long bad = 0;
    for (unsigned long long i = 0; i < (1ull << 32); ++i) {
        const unsigned u = (unsigned)i;
        float f;
        std::memcpy(&f, &u, sizeof f);
        const double want = (double)f;
        const bool special = art::widen_special(f) != 0;
        const bool normal_or_zero = !(std::fpclassify(f) == FP_SUBNORMAL || std::isinf(f) ||
                                      std::isnan(f));
        if (special == normal_or_zero) ++bad;
        if (!special && art::fm_bits(art::widen(f)) != art::fm_bits(want)) ++bad;
    }
    std::printf("%llu\n", bad);
    return 0;
}
"""

EMIT = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <vector_types.h>
#include "art.h"
#include "grid.cuh"
int art_make_devjob(const art_job* job, art::DevJob* J);
void art_make_synch(const art_job* job, art::SynchConstT<double>* S);
int main(int argc, char** argv)
{
    art_job job;
    FILE* fj = std::fopen(argv[1], "rb");
    if (!fj || std::fread(&job, sizeof job, 1, fj) != 1) return 2;
    std::fclose(fj);
    const int n1 = std::atoi(argv[3]), n2 = std::atoi(argv[4]), n3 = std::atoi(argv[5]);
    const double x1min = std::atof(argv[6]), x1max = std::atof(argv[7]);
    std::vector<float4> cells((size_t)2 * n1 * n2 * n3);
    FILE* fg = std::fopen(argv[2], "rb");
    if (!fg || std::fread(cells.data(), sizeof(float4), cells.size(), fg) != cells.size()) return 4;
    std::fclose(fg);
    art::DevJob J;
    if (art_make_devjob(&job, &J)) return 3;
    art::SynchConstT<double> S;
    art_make_synch(&job, &S);
    // the grid part of the device constants, as the library derives them from a loaded grid
    const double me = 9.1093837015e-28, c = 2.99792458e10, mp = 1.67262192369e-24;
    const double pi = 3.14159265358979323846, L3 = job.length_cm * job.length_cm * job.length_cm;
    S.grid = cells.data();
    S.g_n1 = n1;
    S.g_n2 = n2;
    S.g_n3 = n3;
    S.g_x1min = x1min;
    S.g_x1max = x1max;
    S.g_inv_dx1 = n1 / (x1max - x1min);
    S.g_inv_dth = n2 / pi;
    S.g_inv_dph = n3 / (2.0 * pi);
    S.g_gm1 = job.gamma_ad - 1.0;
    S.g_ne_unit = job.m_unit / (L3 * (mp + me));
    S.g_b_unit = c * std::sqrt(4.0 * pi * job.m_unit / L3);
    S.g_th_unit = (mp / me) * (job.gamma_ad - 1.0);
    S.g_r_high = job.r_high;
    S.g_r_low = job.r_low;
    S.g_sigma_cut = job.sigma_cut;
    double v[11];
    while (std::scanf("%lf %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf", v, v + 1, v + 2, v + 3, v + 4,
                      v + 5, v + 6, v + 7, v + 8, v + 9, v + 10) == 11) {
        art::RayState<double> s{v[0], v[1], v[2], v[4], v[5], v[6]};
        const double r = art::ks_radius<double>(v[0], v[1], v[2], J.a2);
        double J4[4], K7[7];
        art::emission_grid<double>(s, r, v[3], J.stokes == 4 ? v + 7 : nullptr, nullptr, J, S, J4,
                                   K7);
        for (int i = 0; i < 4; ++i) std::printf("%.17g ", J4[i]);
        for (int i = 0; i < 7; ++i) std::printf("%.17g ", K7[i]);
        std::printf("\n");
    }
    return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    return None


def _tools():
    gxx, inc = shutil.which("g++"), _cuda_include()
    if gxx is None or inc is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    return gxx, inc


def test_widen_equals_the_conversion_for_every_float(tmp_path):
    gxx, inc = _tools()
    src = tmp_path / "w.cpp"
    src.write_text(WIDEN)
    exe = tmp_path / "w"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert int(out.strip()) == 0


@pytest.mark.parametrize("stokes", [1, 4])
def test_grid_coefficients_match_oracle(tmp_path, stokes):
    from paper_2103_07417_gb300 import art
    gxx, inc = _tools()
    art.load()
    src = tmp_path / "g.cpp"
    src.write_text(EMIT)
    exe = tmp_path / "g"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-I", inc, str(src),
                    "-o", str(exe), "-L", LIBDIR, "-lart_gb300", f"-Wl,-rpath,{LIBDIR}"],
                   check=True)
    snap = W.grmhd_snapshot(seed=0, n1=72, n2=32, n3=32)
    params = {**W.grmhd_8193(n0x=5, n0y=5, levels=0, fov=50.0, stokes=stokes, incl_deg=60.0),
              "precision": "fp64"}
    jfile, gfile = tmp_path / "job.bin", tmp_path / "grid.bin"
    jfile.write_bytes(bytes(art.make_job(**params)))
    gfile.write_bytes(np.ascontiguousarray(snap["data"], np.float32).tobytes())
    oj = O.make_job(grid=snap, **params)
    states = []
    for al, be in [(8.0, 0.0), (-4.0, -4.0), (12.0, 0.0), (-8.0, 0.0), (-12.0, 0.0), (8.0, -4.0),
                   (0.0, -8.0), (12.0, 4.0)]:
        rec, _ = O.trace_record(oj, al, be)
        states.append(rec[:, 1:13])
    y = np.concatenate(states)
    inp = "\n".join(" ".join(f"{v:.17g}" for v in (*row[1:4], row[4], *row[5:8], *row[8:12]))
                    for row in y) + "\n"
    args = [str(exe), str(jfile), str(gfile), str(snap["n1"]), str(snap["n2"]), str(snap["n3"]),
            f"{snap['logr_min']:.17g}", f"{snap['logr_max']:.17g}"]
    out = subprocess.run(args, input=inp, check=True, capture_output=True, text=True).stdout
    got = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    assert got.shape == (len(y), 11)
    want = np.array([np.concatenate(O.coefficients(oj, row, pol=stokes == 4)) for row in y])
    scale = np.abs(want).max(axis=0)
    scale[scale == 0] = 1.0
    err = np.abs(got - want) / scale
    emitting = int((want[:, 0] > 0).sum())
    print("states", len(y), "emitting", emitting, "worst per coefficient", err.max(axis=0))
    assert emitting > 300, emitting
    assert err.max() < 1e-7, err.max(axis=0)
    # and relatively, j_I and alpha_I wherever the emission is not negligible (the Bessel fits'
    # ~1e-7 against the oracle's integrals)
    sel = want[:, 0] > 1e-3 * scale[0]
    for col in (0, 4):
        rel = np.abs(got[sel, col] - want[sel, col]) / np.abs(want[sel, col])
        assert rel.max() < 2e-6, (col, rel.max())
