"""art_trace_pixels_noalloc: the tracer entry point for callers that cannot allocate device
memory (for example a render service whose GPU memory is reserved up front by its own allocator).
It keeps its scratch in one static device array instead of context-allocated buffers; its output
must match art_trace_pixels, call after call, because every call reuses that array.

This file is collected last on purpose, and passes alone in a fresh process as well as after the
other tests."""
import numpy as np
import pytest

from paper_2103_07417_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-6  # the per-pixel tolerance of the other GPU parity tests


def _close(got, ref):
    peak = np.max(np.abs(ref))
    return np.abs(got - ref) <= RTOL * np.maximum(np.abs(ref), 1e-6 * peak)


def test_noalloc_matches_context_tracer_on_consecutive_calls():
    """Unpolarized analytic jobs in FP64 and mixed precision, then the polarized synchrotron disk
    (Stokes I, Q, U, V; its constants are made without a context) in mixed precision with the
    double-float re-trace and in FP64: every plane against the context's tracer, call after
    call on the same static scratch."""
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    cases = [W.schwarzschild_129(a=0.94, incl_deg=17.0, n0x=17, n0y=13, levels=2, precision="fp64"),
             W.schwarzschild_129(a=0.94, incl_deg=17.0, n0x=17, n0y=13, levels=2, precision="mixed"),
             W.kerr_disk_2049(n0x=17, n0y=13, levels=2, precision="mixed_df", crit_band=0.0),
             W.kerr_disk_2049(n0x=17, n0y=13, levels=2, precision="fp64", crit_band=0.0)]
    for params in cases:                      # calls in a row on the same static scratch
        job = art.make_job(**params)
        nx, ny = art.art_image_size(job)
        rng = np.random.default_rng(5)
        pix = torch.from_numpy(rng.permutation(nx * ny).astype(np.int32)).cuda()
        ref, _ = ctx.trace_pixels(job, pix)
        out = torch.full_like(ref, np.nan)
        steps = torch.zeros(pix.numel(), dtype=torch.int32, device="cuda")
        rc = art.art_trace_pixels_noalloc(job, pix, out, aux={"steps": steps})
        assert rc == art.ART_OK, art.art_strerror(rc)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert _close(got[:, 0], want[:, 0]).all()
        # Q, U, V on the scale of the pixel's I
        scale = np.maximum(np.abs(want[:, 0]), 1e-6 * np.abs(want[:, 0]).max())
        for c in range(1, want.shape[1]):
            assert (np.abs(got[:, c] - want[:, c]) <= RTOL * scale).all(), c
        assert (steps.cpu().numpy() > 0).all()
    ctx.close()


def test_noalloc_rejects_more_rays_than_its_scratch():
    from paper_2103_07417_gb300 import art
    job = art.make_job(**W.schwarzschild_129(n0x=1025, n0y=1025, levels=1))   # 2049^2 pixels
    n = art.NOALLOC_MAX_RAYS + 1
    pix = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    assert art.art_trace_pixels_noalloc(job, pix, out) == art.ART_ERR_ARG
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert art.art_trace_pixels_noalloc(job, empty, out[:0]) == art.ART_OK
