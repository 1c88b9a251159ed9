"""TEST INFRASTRUCTURE ONLY: the plain FP64 CPU oracle for adaptive ray tracing.

The oracle is written from Gelles et al. 2021 (arXiv:2103.07417), Sec. 3.2, Eqs. (epabs),
(eprel), Appendix A and Eqs. (interpdef)-(msedef), plus a textbook Kerr-Schild ray tracer for the
intensity function that the paper leaves to ipole (see ``art_oracle.c``).  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.  It shares
no code with the CUDA library (``paper_2103_07417_gb300``) and neither imports the other.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test against closed forms,
the paper's printed power-law ratios, library routines for special cases, or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = [os.path.join(_HERE, "art_oracle.c")]
_lock = threading.Lock()
_lib = None

EMIT_ANALYTIC, EMIT_SYNCH_DISK, EMIT_GRID, EMIT_BLOB = 0, 1, 2, 8
FLOW_KEPLER, FLOW_STATIC = 0, 1
NORM_IBAR_INT, NORM_PEAK = 0, 1
INTERP_LINEAR, INTERP_NEAREST = 0, 1
EDGE_ONESIDED, EDGE_TRACE = 0, 1
RAY_ESCAPED, RAY_CAPTURED, RAY_CAP, RAY_NAN = 0, 1, 2, 3
MASK_UNSET, MASK_TRACED, MASK_INTERP = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available) into oracle/lib/liboracle.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC + [os.path.join(_HERE, "art_oracle.h")])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp] + _SRC
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:] + ["-lm"], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB)
            return _LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


class Job(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("mass", ctypes.c_double), ("r_obs", ctypes.c_double),
        ("incl_deg", ctypes.c_double), ("fov", ctypes.c_double),
        ("n0x", ctypes.c_int), ("n0y", ctypes.c_int), ("levels", ctypes.c_int),
        ("R_rel", ctypes.c_double), ("R_abs", ctypes.c_double),
        ("abs_norm", ctypes.c_int), ("interp", ctypes.c_int), ("edge_mode", ctypes.c_int),
        ("emission", ctypes.c_int), ("flow", ctypes.c_int), ("stokes", ctypes.c_int),
        ("subrings", ctypes.c_int), ("max_steps", ctypes.c_int),
        ("step_frac", ctypes.c_double), ("h_min", ctypes.c_double),
        ("horizon_eps", ctypes.c_double), ("escape_frac", ctypes.c_double),
        ("disk_w", ctypes.c_double), ("blob_sigma", ctypes.c_double),
        ("ne0", ctypes.c_double), ("thetae0", ctypes.c_double), ("b0", ctypes.c_double),
        ("nu_hz", ctypes.c_double), ("ne_slope", ctypes.c_double), ("te_slope", ctypes.c_double),
        ("r_in", ctypes.c_double), ("length_cm", ctypes.c_double),
        ("bz_ratio", ctypes.c_double),
        ("grid", ctypes.POINTER(ctypes.c_float)),
        ("gn1", ctypes.c_int), ("gn2", ctypes.c_int), ("gn3", ctypes.c_int), ("gpad", ctypes.c_int),
        ("glogr_min", ctypes.c_double), ("glogr_max", ctypes.c_double),
        ("gamma_ad", ctypes.c_double), ("m_unit", ctypes.c_double),
        ("r_high", ctypes.c_double), ("r_low", ctypes.c_double), ("sigma_cut", ctypes.c_double),
        ("criterion", ctypes.c_int), ("criterion_plane", ctypes.c_int),
    ]


class RayInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("nturn", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("min_r", ctypes.c_double), ("lam", ctypes.c_double), ("eta", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("rays_traced", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("rays_per_level", ctypes.c_int64 * 16), ("ibar", ctypes.c_double)]


_DEFAULTS = dict(a=0.0, mass=1.0, r_obs=1000.0, incl_deg=60.0, fov=40.0, n0x=33, n0y=33,
                 levels=2, R_rel=0.01, R_abs=1e-4, abs_norm=NORM_IBAR_INT,
                 interp=INTERP_LINEAR, edge_mode=EDGE_ONESIDED, emission=EMIT_ANALYTIC,
                 flow=FLOW_KEPLER, stokes=1, subrings=0, max_steps=100000, step_frac=0.05,
                 h_min=1e-4, horizon_eps=0.01, escape_frac=1.01, disk_w=0.3, blob_sigma=1.0,
                 ne0=0.0, thetae0=0.0, b0=0.0, nu_hz=230e9, ne_slope=-1.1, te_slope=-0.84,
                 r_in=0.0, length_cm=9.6e14, bz_ratio=1.0, gamma_ad=13.0 / 9.0, m_unit=1e27,
                 r_high=20.0, r_low=1.0, sigma_cut=1.0, criterion=0,
                 criterion_plane=0)


_NAMES = dict(
    emission={"analytic": EMIT_ANALYTIC, "synch_disk": EMIT_SYNCH_DISK, "grid": EMIT_GRID,
              "blob": EMIT_BLOB},
    flow={"kepler": FLOW_KEPLER, "static": FLOW_STATIC},
    abs_norm={"ibar_int": NORM_IBAR_INT, "peak": NORM_PEAK},
    interp={"linear": INTERP_LINEAR, "nearest": INTERP_NEAREST},
    edge_mode={"onesided": EDGE_ONESIDED, "trace": EDGE_TRACE},
    criterion={"I": 0, "stokes_any": 1},
)


def make_job(grid=None, **params) -> Job:
    """Build the oracle's job from a parameter dict; option names ("analytic", "peak", ...) are
    mapped to the oracle's enums and keys the oracle does not use are ignored.

    grid: the fluid snapshot for emission "grid", a dict with ``data`` (float32, shape
    (n3, n2, n1, 8)), ``n1``, ``n2``, ``n3``, ``logr_min``, ``logr_max`` (and optionally
    ``gamma``).  The job keeps a reference to the array."""
    d = dict(_DEFAULTS)
    for k, v in params.items():
        if k not in _DEFAULTS:
            continue
        if k in _NAMES and isinstance(v, str):
            v = _NAMES[k][v]
        d[k] = v
    job = Job(**d)
    if grid is not None:
        arr = np.ascontiguousarray(grid["data"], dtype=np.float32)
        n1, n2, n3 = int(grid["n1"]), int(grid["n2"]), int(grid["n3"])
        if arr.shape != (n3, n2, n1, 8):
            raise ValueError("grid data must have shape (n3, n2, n1, 8)")
        job.grid = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        job.gn1, job.gn2, job.gn3 = n1, n2, n3
        job.glogr_min, job.glogr_max = float(grid["logr_min"]), float(grid["logr_max"])
        if "gamma" in grid and "gamma_ad" not in params:
            job.gamma_ad = float(grid["gamma"])
        job._grid_ref = arr
    return job


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            dp, ip64, u8p = P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_uint8)
            lib.orc_image_size.argtypes = [P(Job), P(ctypes.c_int), P(ctypes.c_int)]
            lib.orc_planes.argtypes = [P(Job)]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_trace_screen.argtypes = [P(Job), ctypes.c_int, dp, dp, dp, P(RayInfo)]
            lib.orc_trace_pixels.argtypes = [P(Job), ctypes.c_int, ip64, dp, P(RayInfo)]
            lib.orc_trace_record.argtypes = [P(Job), ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, dp, P(ctypes.c_int)]
            lib.orc_emission.argtypes = [P(Job), dp, dp, dp, dp]
            lib.orc_grid_fluid.argtypes = [P(Job), dp, dp, dp, dp, dp]
            lib.orc_ibar_int.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.orc_ibar_int.restype = ctypes.c_double
            lib.orc_refine_level.argtypes = [P(Job), dp, u8p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, dp, dp]
            lib.orc_render.argtypes = [P(Job), dp, dp, u8p, P(Stats)]
            lib.orc_metrics.argtypes = [dp, dp, u8p, ctypes.c_int, ctypes.c_int, dp]
            lib.orc_bessel_k.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.orc_bessel_k.restype = ctypes.c_double
            lib.orc_synch_coeffs.argtypes = [ctypes.c_double] * 5 + [dp]
            lib.orc_segment.argtypes = [dp, dp, ctypes.c_double, dp, dp]
            lib.orc_transport_rhs.argtypes = [P(Job), dp, dp]
            lib.orc_coefficients.argtypes = [P(Job), dp, ctypes.c_int, dp, dp]
            _lib = lib
    return _lib


def _ptr(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def image_size(job: Job):
    nx, ny = ctypes.c_int(), ctypes.c_int()
    if _load().orc_image_size(ctypes.byref(job), ctypes.byref(nx), ctypes.byref(ny)):
        raise ValueError("invalid grid")
    return nx.value, ny.value


def planes(job: Job) -> int:
    return int(_load().orc_planes(ctypes.byref(job)))


def _info_dict(info):
    return {name: np.array([getattr(x, name) for x in info])
            for name in ("status", "steps", "nturn", "min_r", "lam", "eta")}


def trace_screen(job: Job, alpha, beta):
    """Trace rays at screen points (alpha, beta) [M]; returns (values[n, planes], info dict)."""
    al = np.ascontiguousarray(alpha, dtype=np.float64).ravel()
    be = np.ascontiguousarray(beta, dtype=np.float64).ravel()
    n = al.size
    out = np.zeros((n, planes(job)))
    info = (RayInfo * max(n, 1))()
    rc = _load().orc_trace_screen(ctypes.byref(job), n, _ptr(al), _ptr(be), _ptr(out), info)
    if rc:
        raise RuntimeError(f"orc_trace_screen failed ({rc})")
    return out, _info_dict(info[:n])


def trace_pixels(job: Job, pix):
    """Trace the pixels with linear indices j*nx + i of the final grid."""
    p = np.ascontiguousarray(pix, dtype=np.int64).ravel()
    n = p.size
    out = np.zeros((n, planes(job)))
    info = (RayInfo * max(n, 1))()
    rc = _load().orc_trace_pixels(ctypes.byref(job), n, _ptr(p, ctypes.c_int64), _ptr(out), info)
    if rc:
        raise RuntimeError(f"orc_trace_pixels failed ({rc})")
    return out, _info_dict(info[:n])


def trace_record(job: Job, alpha: float, beta: float, maxrec: int = 200000):
    """Per-step record of one ray: columns (affine lambda, x^mu [1:5], k_mu [5:9],
    f_mu [9:13] (polarization covector, zero when unpolarized), I [13])."""
    rec = np.zeros((maxrec, 14))
    nrec = ctypes.c_int()
    status = _load().orc_trace_record(ctypes.byref(job), alpha, beta, maxrec, _ptr(rec),
                                      ctypes.byref(nrec))
    return rec[: nrec.value].copy(), int(status)


def grid_fluid(job: Job, x):
    """Fluid state of the grid model at Cartesian Kerr-Schild points x (n, 4): returns a dict of
    prim (n, 8) interpolated primitives, u (n, 4), b (n, 4) contravariant, plasma (n, 4) =
    (n_e, Theta_e, |B|, sigma) and emits (n,) bool."""
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    n = x.shape[0]
    prim, u, b, pl = (np.zeros((n, k)) for k in (8, 4, 4, 4))
    em = np.zeros(n, bool)
    lib = _load()
    for i in range(n):
        em[i] = bool(lib.orc_grid_fluid(ctypes.byref(job), _ptr(x[i]), _ptr(prim[i]), _ptr(u[i]),
                                        _ptr(b[i]), _ptr(pl[i])))
    return dict(prim=prim, u=u, b=b, plasma=pl, emits=em)


def emission(job: Job, x, k):
    """Invariant emissivity j/nu^2 and fluid-frame frequency nu = k.u at one point."""
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ka = np.ascontiguousarray(k, dtype=np.float64)
    j, nu = ctypes.c_double(), ctypes.c_double()
    _load().orc_emission(ctypes.byref(job), _ptr(xa), _ptr(ka), ctypes.byref(j), ctypes.byref(nu))
    return j.value, nu.value


def ibar_int(img, stride: int) -> float:
    a = np.ascontiguousarray(img, dtype=np.float64)
    ny, nx = a.shape
    return float(_load().orc_ibar_int(_ptr(a), nx, ny, int(stride)))


def refine_level(job: Job, img, mask, level: int, norm: float):
    """One refinement level in place on copies; returns (img, mask, est_abs, est_rel) (the
    estimates of plane 0).  img: (ny, nx), or (planes, ny, nx) with the job's plane count."""
    a = np.array(img, dtype=np.float64, order="C", copy=True)
    m = np.array(mask, dtype=np.uint8, order="C", copy=True)
    ny, nx = a.shape[-2:]
    if a.ndim == 3 and a.shape[0] != planes(job):
        raise ValueError("img planes do not match the job")
    ea = np.full((ny, nx), np.nan)
    er = np.full((ny, nx), np.nan)
    rc = _load().orc_refine_level(ctypes.byref(job), _ptr(a), _ptr(m, ctypes.c_uint8), nx, ny,
                                  int(level), float(norm), _ptr(ea), _ptr(er))
    if rc:
        raise ValueError(f"orc_refine_level failed ({rc})")
    return a, m, ea, er


def render(job: Job, truth=None):
    """The adaptive scheme; with `truth` (ny x nx, or planes x ny x nx) the tracer is replaced
    by a lookup.  Returns (img [ny x nx, or planes x ny x nx], mask, stats dict)."""
    nx, ny = image_size(job)
    npl = planes(job)
    img = np.zeros((npl, ny, nx))
    mask = np.zeros((ny, nx), dtype=np.uint8)
    st = Stats()
    tp = None
    if truth is not None:
        t = np.ascontiguousarray(truth, dtype=np.float64).reshape(npl, ny, nx)
        tp = _ptr(t)
    rc = _load().orc_render(ctypes.byref(job), tp, _ptr(img), _ptr(mask, ctypes.c_uint8),
                            ctypes.byref(st))
    if rc:
        raise RuntimeError(f"orc_render failed ({rc})")
    stats = dict(rays_traced=st.rays_traced, steps=st.steps, ibar=st.ibar,
                 rays_per_level=[st.rays_per_level[k] for k in range(job.levels + 1)])
    return (img[0] if npl == 1 else img), mask, stats


def bessel_k(n: int, x: float) -> float:
    return float(_load().orc_bessel_k(int(n), float(x)))


def synch_coeffs(ne, thetae, B, nu, theta_b):
    """{j_I, j_Q, j_V, alpha_I, alpha_Q, rho_Q, rho_V} (cgs) in the frame whose Q axis is the
    emission's E-vector."""
    out = np.zeros(7)
    _load().orc_synch_coeffs(float(ne), float(thetae), float(B), float(nu), float(theta_b),
                             _ptr(out))
    return out


def transport_rhs(job: Job, y12):
    """d f_mu / d lambda of the parallel-transported covector for state (x, k, f)."""
    y = np.ascontiguousarray(y12, dtype=np.float64)
    df = np.zeros(4)
    _load().orc_transport_rhs(ctypes.byref(job), _ptr(y), _ptr(df))
    return df


def coefficients(job: Job, y12, pol: bool = True):
    """(J4, K7) emission and absorption/rotation coefficients at state (x, k, f), code units."""
    y = np.ascontiguousarray(y12, dtype=np.float64)
    J4, K7 = np.zeros(4), np.zeros(7)
    _load().orc_coefficients(ctypes.byref(job), _ptr(y), int(pol), _ptr(J4), _ptr(K7))
    return J4, K7


def segment(K7, J4, h):
    """(E, X): exact propagator exp(-K h) and source integral of one constant segment."""
    K = np.ascontiguousarray(K7, dtype=np.float64)
    J = np.ascontiguousarray(J4, dtype=np.float64)
    E = np.zeros(16)
    X = np.zeros(4)
    _load().orc_segment(_ptr(K), _ptr(J), float(h), _ptr(E), _ptr(X))
    return E.reshape(4, 4), X


def metrics(truth, img, mask=None):
    """(IF, FE, MSE, MSE/mean^2) of `img` against `truth` (Eqs. interpdef, fluxdef, msedef)."""
    t = np.ascontiguousarray(truth, dtype=np.float64)
    a = np.ascontiguousarray(img, dtype=np.float64)
    ny, nx = t.shape
    out = np.zeros(4)
    mp = None
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        mp = _ptr(m, ctypes.c_uint8)
    _load().orc_metrics(_ptr(t), _ptr(a), mp, nx, ny, _ptr(out))
    return dict(IF=out[0], FE=out[1], MSE=out[2], MSE_mean=out[3])
