"""Thin ctypes binding of libart_gb300.so (include/art.h).

Argument marshalling only: every step of the adaptive render runs in the library's CUDA
kernels.  Device buffers are torch tensors (PyTorch supplies device memory and the stream).
There is no CPU fallback: if the library cannot be built or loaded, or no CUDA device exists,
these functions raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ART_OK, ART_ERR_ARG, ART_ERR_CUDA, ART_ERR_OOM, ART_ERR_UNSUPPORTED, ART_ERR_DEVICE = (
    0, -1, -2, -3, -4, -5)
MASK_UNSET, MASK_TRACED, MASK_INTERP, MASK_AXIS = 0, 1, 2, 3
RAY_ESCAPED, RAY_CAPTURED, RAY_CAP, RAY_NAN = 0, 1, 2, 3

_NAMES = dict(
    emission={"analytic": 0, "synch_disk": 1, "grid": 2},
    flow={"kepler": 0, "static": 1},
    abs_norm={"ibar_int": 0, "peak": 1},
    interp={"linear": 0, "nearest": 1},
    edge_mode={"onesided": 0, "trace": 1},
    precision={"fp64": 0, "mixed": 1, "fp32": 2, "mixed_df": 3, "mixed_exact": 4},
    criterion={"I": 0, "stokes_any": 1},
)


class Job(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("r_obs", ctypes.c_double), ("incl_deg", ctypes.c_double),
        ("fov", ctypes.c_double), ("n0x", ctypes.c_int32), ("n0y", ctypes.c_int32),
        ("levels", ctypes.c_int32), ("R_rel", ctypes.c_double), ("R_abs", ctypes.c_double),
        ("abs_norm", ctypes.c_int32), ("interp", ctypes.c_int32), ("edge_mode", ctypes.c_int32),
        ("emission", ctypes.c_int32), ("flow", ctypes.c_int32), ("stokes", ctypes.c_int32),
        ("subrings", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("max_steps", ctypes.c_int32), ("fp64_sweep", ctypes.c_double),
        ("step_frac", ctypes.c_double), ("h_min", ctypes.c_double),
        ("horizon_eps", ctypes.c_double), ("escape_frac", ctypes.c_double),
        ("disk_w", ctypes.c_double), ("ne0", ctypes.c_double), ("thetae0", ctypes.c_double),
        ("b0", ctypes.c_double), ("nu_hz", ctypes.c_double), ("ne_slope", ctypes.c_double),
        ("te_slope", ctypes.c_double), ("r_in", ctypes.c_double), ("length_cm", ctypes.c_double),
        ("bz_ratio", ctypes.c_double), ("gamma_ad", ctypes.c_double), ("m_unit", ctypes.c_double),
        ("r_high", ctypes.c_double), ("r_low", ctypes.c_double), ("sigma_cut", ctypes.c_double),
        ("proposal", ctypes.c_int32), ("proposal_depth", ctypes.c_int32),
        ("proposal_p", ctypes.c_double), ("crit_band", ctypes.c_double),
        ("criterion", ctypes.c_int32), ("criterion_plane", ctypes.c_int32),
    ]


class Tune(ctypes.Structure):
    """art_tune: FP32 kernel-form thresholds in rays per block (quad form up to quad_rays, pair
    form up to pair_rays), the persistent grids' blocks per SM of the FP64 and of the FP32 /
    double-float launches (0: as many as fit), and the FP64 launches' quad-form threshold."""
    _fields_ = [("quad_rays", ctypes.c_int32), ("pair_rays", ctypes.c_int32),
                ("blocks64", ctypes.c_int32), ("blocks32", ctypes.c_int32),
                ("quad64_rays", ctypes.c_int32)]


TUNE_DEFAULT = (32, 64, 1, 0, 32)


class Stats(ctypes.Structure):
    _fields_ = [("rays_traced", ctypes.c_int64), ("rays_fp64", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("rays_capped", ctypes.c_int64),
                ("rays_nan", ctypes.c_int64), ("rays_per_level", ctypes.c_int64 * 16),
                ("norm", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("rays_speculative", ctypes.c_int64), ("rays_spec_used", ctypes.c_int64),
                ("rays_exact", ctypes.c_int64), ("border_points", ctypes.c_int64),
                ("border_overflow", ctypes.c_int64)]


class LaunchRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("ms", ctypes.c_float),
                ("steps", ctypes.c_int64), ("items", ctypes.c_int64),
                ("max_steps", ctypes.c_int64)]


KERNEL_KINDS = {0: "trace_fp64", 1: "trace_fp32", 2: "refine", 3: "other", 4: "trace_df",
                5: "propose"}


class RayAux(ctypes.Structure):
    _fields_ = [("status", ctypes.c_void_p), ("steps", ctypes.c_void_p),
                ("nturn", ctypes.c_void_p), ("min_r", ctypes.c_void_p)]


_JOB_DEFAULTS = dict(fp64_sweep=3.0 * 3.141592653589793, gamma_ad=13.0 / 9.0, m_unit=3e26,
                     r_high=20.0, r_low=1.0, sigma_cut=1.0, proposal=0, proposal_depth=2,
                     proposal_p=0.5, crit_band=0.0, criterion=0, criterion_plane=0)


def make_job(**params) -> Job:
    """The library's job from a parameter dict (option names are mapped to the C enums)."""
    d = dict(_JOB_DEFAULTS)
    d.update(params)
    kw = {}
    for name, _ in Job._fields_:
        if name not in d:
            raise KeyError(f"job parameter {name!r} missing")
        v = d[name]
        if name in _NAMES and isinstance(v, str):
            v = _NAMES[name][v]
        kw[name] = v
    return Job(**kw)


_lock = threading.Lock()
_lib = None

EXPORTS = ("art_create", "art_destroy", "art_strerror", "art_image_size", "art_planes",
           "art_trace_pixels", "art_ibar_int", "art_refine_level", "art_render",
           "art_render_host", "art_metrics", "art_profile", "art_profile_read",
           "art_trace_pixels_noalloc", "art_render_batch", "art_load_grid", "art_cnn_load",
           "art_cnn_read", "art_cnn_forward", "art_cnn_grad", "art_cnn_train_step",
           "art_cnn_sample", "art_set_tune", "art_get_tune", "art_autotune", "art_graph_render",
           "art_graph_render_batch", "art_measure_alu_peaks", "art_measure_fp64_issue",
           "art_visibilities",
           "art_render_axis")
CNN_PARAMS = 28673
NOALLOC_MAX_RAYS = 1 << 20


def lib_path() -> str:
    return _build.LIB


def load():
    """Build (if needed) and load libart_gb300.so; raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            P = ctypes.POINTER
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            lib.art_create.argtypes = [P(vp), ctypes.c_int, vp]
            lib.art_destroy.argtypes = [vp]
            lib.art_destroy.restype = None
            lib.art_strerror.argtypes = [ctypes.c_int]
            lib.art_strerror.restype = ctypes.c_char_p
            lib.art_image_size.argtypes = [P(Job), P(i32), P(i32)]
            lib.art_planes.argtypes = [P(Job)]
            lib.art_trace_pixels.argtypes = [vp, P(Job), vp, i64, vp, P(RayAux)]
            lib.art_ibar_int.argtypes = [vp, vp, i32, i32, i32, P(ctypes.c_double),
                                         P(ctypes.c_double)]
            lib.art_refine_level.argtypes = [vp, P(Job), vp, vp, i32, ctypes.c_double, vp, P(i64)]
            lib.art_render.argtypes = [vp, P(Job), vp, vp, vp, P(Stats)]
            lib.art_render_host.argtypes = [vp, P(Job), vp, vp, P(Stats)]
            lib.art_metrics.argtypes = [vp, vp, vp, vp, i32, i32, P(ctypes.c_double)]
            lib.art_profile.argtypes = [vp, ctypes.c_int]
            lib.art_profile_read.argtypes = [vp, P(LaunchRecord), ctypes.c_int, P(ctypes.c_int)]
            lib.art_trace_pixels_noalloc.argtypes = [P(Job), vp, i64, vp, P(RayAux), vp]
            lib.art_render_batch.argtypes = [vp, P(Job), i32, P(vp), P(vp), P(Stats)]
            lib.art_load_grid.argtypes = [vp, vp, i32, i32, i32, ctypes.c_double, ctypes.c_double]
            fp = P(ctypes.c_float)
            lib.art_cnn_load.argtypes = [vp, vp]
            lib.art_cnn_read.argtypes = [vp, vp]
            lib.art_cnn_forward.argtypes = [vp, vp, i32, i32, vp]
            lib.art_cnn_grad.argtypes = [vp, vp, i32, i32, vp, fp, vp]
            lib.art_cnn_train_step.argtypes = [vp, vp, i32, i32, vp, ctypes.c_float, fp]
            lib.art_cnn_sample.argtypes = [vp, P(Job), vp, vp, i32, vp, vp]
            lib.art_set_tune.argtypes = [vp, P(Tune)]
            lib.art_get_tune.argtypes = [vp, P(Tune)]
            lib.art_measure_alu_peaks.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double)]
            lib.art_measure_fp64_issue.argtypes = [vp, P(ctypes.c_double)]
            lib.art_autotune.argtypes = [vp, P(Job), vp, vp, i32, P(Tune), fp]
            lib.art_graph_render.argtypes = [vp, P(Job), vp, vp]
            lib.art_visibilities.argtypes = [vp, vp, vp, i32, i32, ctypes.c_double,
                                             ctypes.c_double, i32, vp]
            lib.art_render_axis.argtypes = [vp, P(Job), i32, i32, ctypes.c_double,
                                            ctypes.c_double, P(vp), P(vp), vp, P(Stats)]
            lib.art_graph_render_batch.argtypes = [vp, P(Job), i32, P(vp), P(vp)]
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != ART_OK:
        msg = load().art_strerror(rc).decode()
        raise RuntimeError(f"{what} failed: {msg} ({rc})")


def art_strerror(code: int) -> str:
    return load().art_strerror(int(code)).decode()


def art_image_size(job: Job):
    nx, ny = ctypes.c_int32(), ctypes.c_int32()
    _check(load().art_image_size(ctypes.byref(job), ctypes.byref(nx), ctypes.byref(ny)),
           "art_image_size")
    return nx.value, ny.value


def art_planes(job: Job) -> int:
    return int(load().art_planes(ctypes.byref(job)))


def _rayaux(aux):
    if aux is None:
        return None
    return RayAux(*[ctypes.c_void_p(aux[k].data_ptr()) if aux.get(k) is not None else None
                    for k in ("status", "steps", "nturn", "min_r")])


def _check_trace_buffers(job: Job, pix, out, aux):
    """The buffers a pixel trace writes must hold what the library writes there: int32 pixels,
    float64 outputs of at least n x planes, int32/float32 aux arrays of at least n."""
    import torch
    n = pix.numel()
    if pix.dtype != torch.int32:
        raise ValueError("pix must be int32")
    if out.dtype != torch.float64 or out.numel() < n * art_planes(job) or not out.is_contiguous():
        raise ValueError("out must be contiguous float64 with at least n x planes elements")
    for k, dt in (("status", torch.int32), ("steps", torch.int32), ("nturn", torch.int32),
                  ("min_r", torch.float32)):
        t = (aux or {}).get(k)
        if t is not None and (t.dtype != dt or t.numel() < n):
            raise ValueError(f"aux[{k!r}] must be {dt} with at least n elements")


def art_trace_pixels_noalloc(job: Job, pix, out, aux: dict | None = None, stream=None) -> int:
    """The allocation-free tracer (no context; current device; `stream` a torch stream or None
    for torch's current stream).  Returns the C return code instead of raising, so callers can
    see the size rejection."""
    import torch
    _check_trace_buffers(job, pix, out, aux)
    s = stream if stream is not None else torch.cuda.current_stream()
    ra = _rayaux(aux)
    return int(load().art_trace_pixels_noalloc(ctypes.byref(job), _dptr(pix), pix.numel(),
                                                _dptr(out), ctypes.byref(ra) if ra else None,
                                                ctypes.c_void_p(s.cuda_stream)))


def _dptr(t):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stats_dict(st: Stats, levels: int) -> dict:
    return dict(rays_traced=st.rays_traced, rays_fp64=st.rays_fp64, steps=st.steps,
                rays_capped=st.rays_capped, rays_nan=st.rays_nan, norm=st.norm,
                kernel_launches=st.kernel_launches, rays_speculative=st.rays_speculative,
                rays_spec_used=st.rays_spec_used, rays_exact=st.rays_exact,
                border_points=st.border_points, border_overflow=st.border_overflow,
                rays_per_level=[st.rays_per_level[k] for k in range(levels + 1)])


class Context:
    """An art_ctx bound to a CUDA device and a torch stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libart_gb300 needs a CUDA device (no CPU fallback)")
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._ctx = ctypes.c_void_p()
        _check(load().art_create(ctypes.byref(self._ctx), device,
                                 ctypes.c_void_p(self.stream.cuda_stream)), "art_create")

    def close(self):
        if self._ctx:
            load().art_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI calls ---------------------------------------------------------------------
    def art_trace_pixels(self, job: Job, pix, out, aux: dict | None = None):
        _check_trace_buffers(job, pix, out, aux)
        ra = None
        if aux is not None:
            ra = RayAux(*[ctypes.c_void_p(aux[k].data_ptr()) if aux.get(k) is not None else None
                          for k in ("status", "steps", "nturn", "min_r")])
        _check(load().art_trace_pixels(self._ctx, ctypes.byref(job), _dptr(pix), pix.numel(),
                                       _dptr(out), ctypes.byref(ra) if ra else None),
               "art_trace_pixels")

    def art_ibar_int(self, img, stride: int):
        ib, pk = ctypes.c_double(), ctypes.c_double()
        ny, nx = img.shape[-2], img.shape[-1]
        _check(load().art_ibar_int(self._ctx, _dptr(img), nx, ny, stride, ctypes.byref(ib),
                                   ctypes.byref(pk)), "art_ibar_int")
        return ib.value, pk.value

    def art_refine_level(self, job: Job, img, mask, level: int, norm: float, queue) -> int:
        n = ctypes.c_int64()
        _check(load().art_refine_level(self._ctx, ctypes.byref(job), _dptr(img), _dptr(mask),
                                       level, norm, _dptr(queue), ctypes.byref(n)),
               "art_refine_level")
        return n.value

    def art_render(self, job: Job, img, mask=None, truth=None, stats: bool = True):
        st = Stats()
        _check(load().art_render(self._ctx, ctypes.byref(job), _dptr(truth), _dptr(img),
                                 _dptr(mask), ctypes.byref(st) if stats else None), "art_render")
        return _stats_dict(st, job.levels) if stats else None

    def art_render_batch(self, jobs, imgs, masks=None, stats: bool = True):
        n = len(jobs)
        jarr = (Job * n)(*jobs)
        iarr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in imgs])
        marr = (ctypes.c_void_p * n)(*[m.data_ptr() for m in masks]) if masks is not None else None
        st = (Stats * n)()
        _check(load().art_render_batch(self._ctx, jarr, n, iarr, marr, st if stats else None),
               "art_render_batch")
        return [_stats_dict(st[i], jobs[i].levels) for i in range(n)] if stats else None

    def art_graph_render_batch(self, jobs, imgs, masks=None):
        """art_render_batch through a CUDA graph captured on the first call for this batch."""
        n = len(jobs)
        jarr = (Job * n)(*jobs)
        iarr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in imgs])
        marr = (ctypes.c_void_p * n)(*[m.data_ptr() for m in masks]) if masks is not None else None
        _check(load().art_graph_render_batch(self._ctx, jarr, n, iarr, marr),
               "art_graph_render_batch")

    def render_batch(self, jobs):
        """Allocate the images and masks of a batch on the device and run art_render_batch."""
        import torch
        imgs, masks = [], []
        for j in jobs:
            nx, ny = art_image_size(j)
            imgs.append(torch.empty((art_planes(j), ny, nx), dtype=torch.float64,
                                    device=f"cuda:{self.device}"))
            masks.append(torch.empty((ny, nx), dtype=torch.uint8, device=f"cuda:{self.device}"))
        stats = self.art_render_batch(jobs, imgs, masks)
        return imgs, masks, stats

    def art_render_host(self, job: Job, img: np.ndarray, mask: np.ndarray | None = None):
        st = Stats()
        assert img.flags.c_contiguous and img.dtype == np.float64
        mp = mask.ctypes.data_as(ctypes.c_void_p) if mask is not None else None
        _check(load().art_render_host(self._ctx, ctypes.byref(job),
                                      img.ctypes.data_as(ctypes.c_void_p), mp, ctypes.byref(st)),
               "art_render_host")
        return _stats_dict(st, job.levels)

    def art_metrics(self, truth, img, mask=None) -> dict:
        out = (ctypes.c_double * 4)()
        ny, nx = truth.shape[-2], truth.shape[-1]
        _check(load().art_metrics(self._ctx, _dptr(truth), _dptr(img), _dptr(mask), nx, ny, out),
               "art_metrics")
        return dict(IF=out[0], FE=out[1], MSE=out[2], MSE_mean=out[3])

    def art_load_grid(self, grid, n1: int, n2: int, n3: int, logr_min: float, logr_max: float):
        """Load the fluid snapshot of grid jobs: a contiguous float32 CUDA tensor (referenced; the
        context keeps a Python reference) or a numpy array (copied), shape (n3, n2, n1, 8)."""
        if grid is None:
            ptr = None
        elif isinstance(grid, np.ndarray):
            if not (grid.flags.c_contiguous and grid.dtype == np.float32):
                raise ValueError("grid must be a contiguous float32 array")
            ptr = grid.ctypes.data_as(ctypes.c_void_p)
        else:
            import torch
            if grid.dtype != torch.float32:
                raise ValueError("grid must be float32")
            ptr = _dptr(grid)
        _check(load().art_load_grid(self._ctx, ptr, int(n1), int(n2), int(n3), float(logr_min),
                                    float(logr_max)), "art_load_grid")
        self._grid_ref = grid if (grid is not None and not isinstance(grid, np.ndarray)) else None

    def load_grid(self, snap: dict, on_device: bool = True):
        """Load a snapshot dict (data, n1, n2, n3, logr_min, logr_max), by default as a device
        tensor."""
        data = snap["data"]
        if on_device:
            import torch
            data = torch.from_numpy(np.ascontiguousarray(data, np.float32)).to(f"cuda:{self.device}")
        self.art_load_grid(data, snap["n1"], snap["n2"], snap["n3"], snap["logr_min"],
                           snap["logr_max"])

    # -- learned block proposal ----------------------------------------------------------------
    def art_cnn_load(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        if p.size != CNN_PARAMS:
            raise ValueError(f"expected {CNN_PARAMS} parameters")
        _check(load().art_cnn_load(self._ctx, p.ctypes.data_as(ctypes.c_void_p)), "art_cnn_load")

    def art_cnn_read(self) -> np.ndarray:
        p = np.empty(CNN_PARAMS, dtype=np.float32)
        _check(load().art_cnn_read(self._ctx, p.ctypes.data_as(ctypes.c_void_p)), "art_cnn_read")
        return p

    @staticmethod
    def cnn_out_shape(H: int, W: int):
        o = lambda n: ((n - 1) // 2 + 1 - 1) // 2 + 1
        return o(H), o(W)

    def art_cnn_forward(self, feat):
        """feat: contiguous float32 CUDA tensor (H, W, 3); returns the (Ho, Wo) probabilities."""
        import torch
        H, W = int(feat.shape[0]), int(feat.shape[1])
        prob = torch.empty(self.cnn_out_shape(H, W), dtype=torch.float32, device=feat.device)
        _check(load().art_cnn_forward(self._ctx, _dptr(feat), H, W, _dptr(prob)), "art_cnn_forward")
        return prob

    def art_cnn_grad(self, feat, target):
        H, W = int(feat.shape[0]), int(feat.shape[1])
        loss = ctypes.c_float()
        g = np.empty(CNN_PARAMS, dtype=np.float32)
        _check(load().art_cnn_grad(self._ctx, _dptr(feat), H, W, _dptr(target), ctypes.byref(loss),
                                   g.ctypes.data_as(ctypes.c_void_p)), "art_cnn_grad")
        return loss.value, g

    def art_cnn_train_step(self, feat, target, lr: float) -> float:
        H, W = int(feat.shape[0]), int(feat.shape[1])
        loss = ctypes.c_float()
        _check(load().art_cnn_train_step(self._ctx, _dptr(feat), H, W, _dptr(target), float(lr),
                                         ctypes.byref(loss)), "art_cnn_train_step")
        return loss.value

    def art_cnn_sample(self, job: Job, img, mask, level: int):
        """(features (H, W, 3), targets (Ho, Wo)) of one level of the context's last render."""
        import torch
        s = 1 << (job.levels - level)
        nx, ny = art_image_size(job)
        H, W = (ny - 1) // s + 1, (nx - 1) // s + 1
        feat = torch.empty((H, W, 3), dtype=torch.float32, device=img.device)
        tgt = torch.empty(self.cnn_out_shape(H, W), dtype=torch.float32, device=img.device)
        _check(load().art_cnn_sample(self._ctx, ctypes.byref(job), _dptr(img), _dptr(mask), level,
                                     _dptr(feat), _dptr(tgt)), "art_cnn_sample")
        return feat, tgt

    def art_graph_render(self, job: Job, img, mask):
        """art_render through a CUDA graph captured on the first call for this job and buffers."""
        _check(load().art_graph_render(self._ctx, ctypes.byref(job), _dptr(img), _dptr(mask)),
               "art_graph_render")

    def art_set_tune(self, quad_rays: int | None = None, pair_rays: int | None = None,
                     blocks64: int = 1, blocks32: int = 0, quad64_rays: int = 32):
        """Set the scheduling (FP32 kernel-form thresholds, grid blocks per SM, FP64 quad-form
        threshold); no arguments restore the defaults."""
        if quad_rays is None and pair_rays is None:
            _check(load().art_set_tune(self._ctx, None), "art_set_tune")
            return
        t = Tune(int(quad_rays), int(pair_rays), int(blocks64), int(blocks32), int(quad64_rays))
        _check(load().art_set_tune(self._ctx, ctypes.byref(t)), "art_set_tune")

    def art_get_tune(self) -> tuple:
        """(quad_rays, pair_rays, blocks64, blocks32, quad64_rays)."""
        t = Tune()
        _check(load().art_get_tune(self._ctx, ctypes.byref(t)), "art_get_tune")
        return t.quad_rays, t.pair_rays, t.blocks64, t.blocks32, t.quad64_rays

    def art_autotune(self, job: Job, img, mask, reps: int = 3):
        """Time `job` under each candidate setting, keep the fastest in the context; returns
        ((quad_rays, pair_rays, blocks64, blocks32, quad64_rays), median ms)."""
        t = Tune()
        ms = ctypes.c_float()
        _check(load().art_autotune(self._ctx, ctypes.byref(job), _dptr(img), _dptr(mask), int(reps),
                                   ctypes.byref(t), ctypes.byref(ms)), "art_autotune")
        return (t.quad_rays, t.pair_rays, t.blocks64, t.blocks32, t.quad64_rays), ms.value

    def art_measure_alu_peaks(self) -> dict:
        """Measured FP32 and FP64 fused multiply-add throughput of this GPU, TFLOP/s."""
        f32, f64 = ctypes.c_double(), ctypes.c_double()
        _check(load().art_measure_alu_peaks(self._ctx, ctypes.byref(f32), ctypes.byref(f64)),
               "art_measure_alu_peaks")
        return {"fp32_tflops": f32.value, "fp64_tflops": f64.value}

    def art_measure_fp64_issue(self) -> dict:
        """SM cycles per FP64 fused multiply-add: one warp with one dependent chain, one warp with
        eight independent chains, and four warps (one per scheduler) per instruction of the SM."""
        c = (ctypes.c_double * 3)()
        _check(load().art_measure_fp64_issue(self._ctx, c), "art_measure_fp64_issue")
        return {"one_warp_chain": c[0], "one_warp_8_chains": c[1], "four_warps_per_sm": c[2]}

    def art_visibilities(self, img, dx: float, taper_fwhm: float, m: int, ref=None, out=None):
        """Visibilities of one image plane (ny, nx) float64 CUDA tensor (minus `ref` if given):
        an (m, m) complex128 tensor, row k_v, column k_u, frequency k stored at k mod m."""
        import torch
        if img.dtype != torch.float64 or img.dim() != 2 or not img.is_contiguous():
            raise ValueError("img must be a contiguous 2-D float64 tensor")
        if ref is not None and (ref.shape != img.shape or ref.dtype != torch.float64
                                or not ref.is_contiguous()):
            raise ValueError("ref must match img")
        ny, nx = int(img.shape[0]), int(img.shape[1])
        if out is None:
            out = torch.empty((m, m, 2), dtype=torch.float64, device=img.device)
        elif out.dtype != torch.float64 or out.numel() < 2 * m * m or not out.is_contiguous():
            raise ValueError("out must hold m x m complex float64 values")
        _check(load().art_visibilities(self._ctx, _dptr(img), _dptr(ref), nx, ny, float(dx),
                                       float(taper_fwhm), int(m), _dptr(out)), "art_visibilities")
        return torch.view_as_complex(out.view(m, m, 2))

    def art_render_axis(self, jobs, levels3: int, R_rel3: float, R_abs3: float, imgs,
                        amask=None, truth=None):
        """Adaptive sampling along a third axis (frequency or time): jobs[f] per sample, imgs a
        list of F device images (planes, ny, nx) float64 (written), amask (optional) an
        (F, ny, nx) uint8 device tensor, truth (optional) a list of F device images.  Returns
        the per-sample stats."""
        import torch
        n = len(jobs)
        if len(imgs) != n or (truth is not None and len(truth) != n):
            raise ValueError("one image (and truth image) per job")
        for t in list(imgs) + list(truth or []):
            if t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("images must be contiguous float64")
        if amask is not None and (amask.dtype != torch.uint8 or amask.numel() < n * imgs[0][0].numel()):
            raise ValueError("amask must be uint8 with F x ny x nx elements")
        jarr = (Job * n)(*jobs)
        iarr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in imgs])
        tarr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in truth]) if truth is not None else None
        st = (Stats * n)()
        _check(load().art_render_axis(self._ctx, jarr, n, int(levels3), float(R_rel3),
                                      float(R_abs3), tarr, iarr, _dptr(amask), st),
               "art_render_axis")
        return [_stats_dict(st[i], jobs[i].levels) for i in range(n)]

    def art_profile(self, enable: bool):
        _check(load().art_profile(self._ctx, int(bool(enable))), "art_profile")

    def art_profile_read(self, cap: int = 256):
        recs = (LaunchRecord * cap)()
        n = ctypes.c_int()
        _check(load().art_profile_read(self._ctx, recs, cap, ctypes.byref(n)), "art_profile_read")
        return [dict(kind=KERNEL_KINDS.get(r.kind, "other"), level=r.level, ms=r.ms, steps=r.steps,
                     items=r.items, max_steps=r.max_steps) for r in recs[: n.value]]

    # -- conveniences ----------------------------------------------------------------------
    def render(self, job: Job, truth=None):
        """Allocate the image and mask on the device and run art_render."""
        import torch
        nx, ny = art_image_size(job)
        planes = art_planes(job)
        img = torch.empty((planes, ny, nx), dtype=torch.float64, device=f"cuda:{self.device}")
        mask = torch.empty((ny, nx), dtype=torch.uint8, device=f"cuda:{self.device}")
        stats = self.art_render(job, img, mask, truth)
        return img, mask, stats

    def trace_pixels(self, job: Job, pix):
        import torch
        planes = art_planes(job)
        out = torch.empty((pix.numel(), planes), dtype=torch.float64, device=pix.device)
        aux = dict(status=torch.empty(pix.numel(), dtype=torch.int32, device=pix.device),
                   steps=torch.empty(pix.numel(), dtype=torch.int32, device=pix.device),
                   nturn=torch.empty(pix.numel(), dtype=torch.int32, device=pix.device),
                   min_r=torch.empty(pix.numel(), dtype=torch.float32, device=pix.device))
        self.art_trace_pixels(job, pix, out, aux)
        return out, aux
