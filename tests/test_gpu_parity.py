"""GPU parity: the CUDA library (through its C-ABI) against the CPU oracle, element by element,
on the same seeded inputs.

Tolerances (the FP64 path computes the same discretisation in a different operation order):
  - traced intensities: |dI| <= 1e-6 max(|I|, 1e-6 I_peak) per pixel;
  - refinement on identical inputs: masks identical and interpolants bit-identical, except points
    whose estimate lies within 1e-9 of the tolerance;
  - full renders: masks may differ only where the oracle's estimate is within 1e-9 (relative) of
    the tolerance, on at most 2 points; all other pixels within the intensity tolerance;
  - ray status and RK4 step counts equal on every ray off the near-critical band.
"""
import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    yield c
    c.close()


def _art():
    from paper_2103_07417_gb300 import art
    return art


def _close(gpu, ref, rtol=RTOL):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    peak = np.max(np.abs(ref)) if ref.size else 0.0
    tol = rtol * np.maximum(np.abs(ref), 1e-6 * peak)
    bad = np.abs(gpu - ref) > tol
    return bad


# ------------------------------------------------------------------------------------------
# tracer
# ------------------------------------------------------------------------------------------

TRACE_CASES = [
    ("schwarzschild_129", W.schwarzschild_129(n0x=17, n0y=17, levels=2)),                             # 65 x 65 grid
    ("kerr17", W.schwarzschild_129(a=0.94, incl_deg=17.0, n0x=13, n0y=11, levels=2)),    # ragged 49 x 41
    ("kerr_retro", W.schwarzschild_129(a=-0.7, incl_deg=75.0, n0x=9, n0y=9, levels=2, fov=24.0)),
    ("static", W.schwarzschild_129(a=0.5, incl_deg=45.0, n0x=9, n0y=9, levels=2, flow="static")),
]


@pytest.mark.parametrize("name,params", TRACE_CASES, ids=[c[0] for c in TRACE_CASES])
def test_trace_pixels_fp64_matches_oracle(ctx, name, params, near_critical):
    art = _art()
    job = art.make_job(**params)
    nx, ny = art.art_image_size(job)
    pix = np.arange(nx * ny, dtype=np.int32)
    pix_d = torch.from_numpy(pix).cuda()
    out, aux = ctx.trace_pixels(job, pix_d)
    torch.cuda.synchronize()
    ref, info = O.trace_pixels(O.make_job(**params), pix.astype(np.int64))
    bad = _close(out.cpu().numpy()[:, 0], ref[:, 0])
    assert bad.sum() == 0, (name, np.flatnonzero(bad)[:10])
    st = aux["status"].cpu().numpy()
    steps = aux["steps"].cpu().numpy()
    # status and RK4 steps equal on every ray off the near-critical band (there the photon
    # shell's instability amplifies the two programs' rounding differences)
    nc = near_critical(params["a"], info)
    ok = ~nc
    print(name, "near-critical rays", int(nc.sum()), "of", len(nc))
    assert (st[ok] == info["status"][ok]).all(), np.flatnonzero(ok & (st != info["status"]))[:10]
    assert (steps[ok] == info["steps"][ok]).all(), np.flatnonzero(ok & (steps != info["steps"]))[:10]
    assert np.all(np.isin(st, [art.RAY_ESCAPED, art.RAY_CAPTURED]))


def test_trace_pixels_empty_and_bad_index(ctx):
    art = _art()
    job = art.make_job(**W.schwarzschild_129(n0x=5, n0y=5, levels=1))
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    out = torch.empty((0, 1), dtype=torch.float64, device="cuda")
    ctx.art_trace_pixels(job, empty, out)
    bad = torch.tensor([0, 10**6], dtype=torch.int32, device="cuda")
    out2 = torch.zeros((2, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        ctx.art_trace_pixels(job, bad, out2)


# ------------------------------------------------------------------------------------------
# refinement kernels on identical inputs
# ------------------------------------------------------------------------------------------

def _level_input(truth, levels, level):
    sprev = 1 << (levels - level + 1)
    img = np.full_like(truth, np.nan)
    img[::sprev, ::sprev] = truth[::sprev, ::sprev]
    mask = np.zeros(truth.shape, np.uint8)
    mask[::sprev, ::sprev] = 1
    return img, mask


REFINE_CASES = [
    dict(n0x=17, n0y=17, levels=3, kind="ring", interp="linear", edge_mode="onesided"),
    dict(n0x=13, n0y=7, levels=3, kind="smooth", interp="linear", edge_mode="trace"),
    dict(n0x=9, n0y=21, levels=2, kind="noisy", interp="nearest", edge_mode="onesided"),
    dict(n0x=33, n0y=1, levels=3, kind="noisy", interp="linear", edge_mode="onesided"),
    dict(n0x=3, n0y=3, levels=4, kind="ring", interp="linear", edge_mode="onesided"),
    # wide exactly uniform regions (zero background, a constant plateau) next to structure:
    # the kernel's uniform-stencil exit must give the FP64 decisions and interpolants
    dict(n0x=17, n0y=17, levels=3, kind="plateau", interp="linear", edge_mode="onesided"),
    dict(n0x=17, n0y=13, levels=3, kind="plateau", interp="linear", edge_mode="trace"),
]


def _image(kind, nx, ny, seed):
    if kind == "ring":
        return W.ring_image(seed, nx, ny)
    if kind == "plateau":
        img = W.ring_image(seed, nx, ny)
        img[img < np.quantile(img, 0.6)] = 0.0
        img[: ny // 3, : nx // 3] = 0.37
        return img
    if kind == "smooth":
        return W.smooth_image(seed, nx, ny)
    return W.smooth_image(seed, nx, ny, noise=0.05)


@pytest.mark.parametrize("case", REFINE_CASES, ids=lambda c: f"{c['n0x']}x{c['n0y']}_{c['kind']}")
def test_refine_level_matches_oracle(ctx, case):
    art = _art()
    params = W.job(n0x=case["n0x"], n0y=case["n0y"], levels=case["levels"], R_abs=2e-3,
                   R_rel=5e-3, interp=case["interp"], edge_mode=case["edge_mode"])
    job = art.make_job(**params)
    ojob = O.make_job(**params)
    nx, ny = art.art_image_size(job)
    truth = _image(case["kind"], nx, ny, seed=case["n0x"] * 7 + case["n0y"])
    norm = float(np.mean(truth))
    for level in range(1, case["levels"] + 1):
        img, mask = _level_input(truth, case["levels"], level)
        ref_img, ref_mask, ea, er = O.refine_level(ojob, img, mask, level, norm)
        img_d = torch.from_numpy(img).cuda()
        mask_d = torch.from_numpy(mask).cuda()
        queue = torch.full((nx * ny,), -1, dtype=torch.int32, device="cuda")
        n = ctx.art_refine_level(job, img_d, mask_d, level, norm, queue)
        gm = mask_d.cpu().numpy()
        gi = img_d.cpu().numpy()
        near = ((np.abs(ea - params["R_abs"]) <= 1e-9 * params["R_abs"])
                | (np.abs(er - params["R_rel"]) <= 1e-9 * params["R_rel"]))
        diff = (gm != ref_mask) & ~near
        assert diff.sum() == 0, (level, np.argwhere(diff)[:5])
        interp = (ref_mask == 2) & (gm == 2)
        np.testing.assert_array_equal(gi[interp], ref_img[interp])
        q = np.sort(queue.cpu().numpy()[:n])
        expect = np.sort(np.flatnonzero((gm == 1).ravel() & np.isnan(img.ravel())))
        np.testing.assert_array_equal(q, expect)
        assert len(np.unique(q)) == n


SCREEN_CASES = ["wide_range", "below_fp32", "quantile_thresholds", "signed_planes"]


@pytest.mark.parametrize("kind", SCREEN_CASES)
def test_refine_fp32_screen_keeps_fp64_decisions(ctx, kind):
    """The refinement kernel decides most points with an FP32 screen of the estimate and falls
    back to FP64 near the thresholds: its masks must equal the oracle's FP64 decisions except
    for estimates within 1e-12 of a tolerance, on images built to stress the screen: magnitudes
    spanning 1e-300 .. 1e30, values below the FP32 range, tolerances placed at quantiles of the
    estimates (many points just above / below them), and signed values."""
    art = _art()
    rng = np.random.default_rng(SCREEN_CASES.index(kind) + 11)
    n0, levels = 17, 3
    params = W.job(n0x=n0, n0y=n0, levels=levels, R_abs=2e-3, R_rel=5e-3)
    nx = ny = (1 << levels) * (n0 - 1) + 1
    if kind == "wide_range":
        truth = 10.0 ** rng.uniform(-300, 30, (ny, nx))
    elif kind == "below_fp32":
        truth = 1e-40 * W.smooth_image(3, nx, ny)
    elif kind == "signed_planes":
        truth = W.smooth_image(4, nx, ny, noise=0.2) - 0.5
    else:
        truth = W.ring_image(5, nx, ny)
    for level in range(1, levels + 1):
        img, mask = _level_input(truth, levels, level)
        norm = float(np.mean(np.abs(truth)))
        if kind == "quantile_thresholds":
            _, _, ea0, er0 = O.refine_level(O.make_job(**params), img, mask, level, norm)
            fin = np.isfinite(ea0) & np.isfinite(er0) & (ea0 > 0)
            params = {**params, "R_abs": float(np.quantile(ea0[fin], 0.4)),
                      "R_rel": float(np.quantile(er0[fin], 0.3))}
        ref_img, ref_mask, ea, er = O.refine_level(O.make_job(**params), img, mask, level, norm)
        img_d = torch.from_numpy(img).cuda()
        mask_d = torch.from_numpy(mask).cuda()
        queue = torch.full((nx * ny,), -1, dtype=torch.int32, device="cuda")
        ctx.art_refine_level(art.make_job(**params), img_d, mask_d, level, norm, queue)
        gm = mask_d.cpu().numpy()
        near = ((np.abs(ea - params["R_abs"]) <= 1e-12 * abs(params["R_abs"]))
                | (np.abs(er - params["R_rel"]) <= 1e-12 * abs(params["R_rel"])))
        diff = (gm != ref_mask) & ~near
        assert diff.sum() == 0, (kind, level, np.argwhere(diff)[:5])
        interp = (ref_mask == 2) & (gm == 2)
        np.testing.assert_array_equal(img_d.cpu().numpy()[interp], ref_img[interp])


def test_ibar_int_matches_oracle(ctx):
    for (nx0, ny0, stride, seed) in [(17, 17, 8, 1), (13, 5, 4, 2), (2, 2, 1, 3), (65, 33, 16, 4)]:
        nx, ny = (nx0 - 1) * stride + 1, (ny0 - 1) * stride + 1
        img = W.smooth_image(seed, nx, ny)
        ib, pk = ctx.art_ibar_int(torch.from_numpy(img).cuda(), stride)
        assert ib == pytest.approx(O.ibar_int(img, stride), rel=1e-14)
        assert pk == np.max(img[::stride, ::stride])


@pytest.mark.parametrize("levels,n0", [(0, 9), (1, 9), (3, 17), (4, 5)])
def test_render_on_truth_matches_oracle(ctx, levels, n0):
    """The whole level loop with 'tracing' replaced by a lookup in a precomputed image."""
    art = _art()
    params = W.job(n0x=n0, n0y=n0 + 2, levels=levels, R_abs=1e-3, R_rel=1e-3)
    job = art.make_job(**params)
    nx, ny = art.art_image_size(job)
    truth = W.ring_image(levels * 10 + n0, nx, ny)
    img, mask, st = ctx.render(job, truth=torch.from_numpy(truth).cuda().reshape(1, ny, nx))
    ref_img, ref_mask, ref_st = O.render(O.make_job(**params), truth)
    np.testing.assert_array_equal(mask.cpu().numpy(), ref_mask)
    np.testing.assert_array_equal(img.cpu().numpy()[0], ref_img)
    assert st["rays_per_level"] == ref_st["rays_per_level"]
    assert st["norm"] == pytest.approx(ref_st["ibar"], rel=1e-14)


# ------------------------------------------------------------------------------------------
# the full adaptive render
# ------------------------------------------------------------------------------------------

RENDER_CASES = [
    ("schwarzschild_129", W.schwarzschild_129()),                                                      # 33^2 -> 129^2
    ("kerr17_ragged", W.schwarzschild_129(a=0.94, incl_deg=17.0, n0x=21, n0y=17, levels=2, R_rel=1e-3,
                             R_abs=1e-3, abs_norm="ibar_int")),
]


@pytest.mark.parametrize("name,params", RENDER_CASES, ids=[c[0] for c in RENDER_CASES])
def test_render_fp64_matches_oracle(ctx, name, params):
    art = _art()
    job = art.make_job(**params)
    img, mask, st = ctx.render(job)
    gi, gm = img.cpu().numpy()[0], mask.cpu().numpy()
    oj = O.make_job(**params)
    ref_img, ref_mask, ref_st = O.render(oj, None)
    assert abs(st["norm"] - ref_st["ibar"]) <= 1e-12 * abs(ref_st["ibar"])
    same = gm == ref_mask
    print(name, "mask differences", int((~same).sum()))
    if not same.all():
        # decisions may differ only where the oracle's estimate is within 1e-9 of a tolerance (observed: none)
        _, _, ea, er = _estimates_at_final(oj, ref_img, ref_mask, ref_st["ibar"])
        d = ~same
        dist = np.minimum(np.abs(ea[d] / oj.R_abs - 1.0), np.abs(er[d] / oj.R_rel - 1.0))
        print(name, "relative distance of the oracle's estimates from a tolerance", dist)
        assert (dist <= 1e-9).all(), name
    assert (~same).sum() <= 2
    bad = _close(gi[same], ref_img[same])
    assert bad.sum() == 0, name
    assert abs(st["rays_traced"] - ref_st["rays_traced"]) <= (~same).sum()


def _estimates_at_final(oj, img, mask, norm):
    """Oracle estimates of every new point of every level, recomputed from the oracle image."""
    ea = np.full(img.shape, np.nan)
    er = np.full(img.shape, np.nan)
    for level in range(1, oj.levels + 1):
        sprev = 1 << (oj.levels - level + 1)
        lvl = np.full_like(img, np.nan)
        lvl[::sprev, ::sprev] = img[::sprev, ::sprev]
        m = np.zeros_like(mask)
        _, _, a, r = O.refine_level(oj, lvl, m, level, norm)
        sel = ~np.isnan(a)
        ea[sel] = a[sel]
        er[sel] = r[sel]
    return None, None, ea, er


def test_render_host_equals_device(ctx):
    art = _art()
    job = art.make_job(**W.schwarzschild_129(n0x=9, n0y=9, levels=2))
    img, mask, st = ctx.render(job)
    nx, ny = art.art_image_size(job)
    himg = np.zeros((1, ny, nx))
    hmask = np.zeros((ny, nx), np.uint8)
    st2 = ctx.art_render_host(job, himg, hmask)
    np.testing.assert_array_equal(himg, img.cpu().numpy())
    np.testing.assert_array_equal(hmask, mask.cpu().numpy())
    assert st2["rays_traced"] == st["rays_traced"]


def test_metrics_match_oracle(ctx):
    truth = W.ring_image(3, 257, 129)
    img = truth + 0.01 * W.smooth_image(4, 257, 129)
    mask = (np.arange(truth.size).reshape(truth.shape) % 3 == 0).astype(np.uint8) * 2
    g = ctx.art_metrics(torch.from_numpy(truth).cuda(), torch.from_numpy(img).cuda(),
                        torch.from_numpy(mask).cuda())
    r = O.metrics(truth, img, mask)
    for k in ("IF", "FE", "MSE", "MSE_mean"):
        assert g[k] == pytest.approx(r[k], rel=1e-12), k


# ------------------------------------------------------------------------------------------
# mixed precision
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["mixed", "mixed_df", "fp32"])
def test_mixed_precision_error_bound(ctx, precision):
    """FP32 geodesics with a high-precision re-trace (FP64 or double-float) of the rays that
    swept >= 3 pi, and plain FP32: the image MSE relative to the mean intensity squared stays
    below 1e-5 against the FP64 oracle (every pixel traced)."""
    art = _art()
    params = W.schwarzschild_129(a=0.94, incl_deg=17.0, n0x=17, n0y=17, levels=2, R_rel=-1.0, R_abs=-1.0)
    job = art.make_job(**{**params, "precision": precision})
    img, mask, st = ctx.render(job)
    ref, _, _ = O.render(O.make_job(**params), None)
    g = img.cpu().numpy()[0]
    mse_mean = np.sum((g - ref) ** 2) / (g.size * np.mean(ref) ** 2)
    assert mse_mean < 1e-5
    assert st["rays_traced"] == g.size
    if precision != "fp32":
        assert st["rays_fp64"] > 0


@pytest.mark.parametrize("geom", [dict(a=0.94, incl_deg=17.0), dict(a=-0.7, incl_deg=75.0)])
def test_double_float_retrace_per_pixel(ctx, geom):
    """Every ray routed to the double-float re-trace (threshold 1e-9 rad): the geodesic carries
    ~48 bits, emission and transfer run in FP32, so each pixel matches the FP64 oracle to 2e-5."""
    art = _art()
    params = W.schwarzschild_129(n0x=13, n0y=13, levels=2, **geom)
    job = art.make_job(**{**params, "precision": "mixed_df", "fp64_sweep": 1e-9})
    nx, ny = art.art_image_size(job)
    pix = np.arange(nx * ny, dtype=np.int32)
    out, aux = ctx.trace_pixels(job, torch.from_numpy(pix).cuda())
    ref, info = O.trace_pixels(O.make_job(**params), pix.astype(np.int64))
    bad = _close(out.cpu().numpy()[:, 0], ref[:, 0], rtol=2e-5)
    assert bad.sum() == 0, np.flatnonzero(bad)[:10]
    st = aux["status"].cpu().numpy()
    assert (st == info["status"]).mean() > 0.995


# ------------------------------------------------------------------------------------------
# the benchmark's own workload at full size (sampled against the oracle)
# ------------------------------------------------------------------------------------------

def _level_of(i, j, levels):
    for k in range(1, levels + 1):
        s = 1 << (levels - k)
        if i % s == 0 and j % s == 0:
            return k, s
    return None, None


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_df"])
def test_bench_workload_sampled(ctx, precision):
    """129^2 -> 2049^2 over 4 levels, exactly as bench.py renders it: sampled traced pixels are
    re-traced by the oracle; sampled interpolated pixels must equal the mean of their 2 or 4
    previous-level neighbours; level counts add up."""
    art = _art()
    params = W.kerr_analytic_2049(precision=precision)
    job = art.make_job(**params)
    img, mask, st = ctx.render(job)
    g = img.cpu().numpy()[0]
    m = mask.cpu().numpy()
    ny, nx = g.shape
    assert (m[::16, ::16] == art.MASK_TRACED).all()
    assert set(np.unique(m)) <= {art.MASK_TRACED, art.MASK_INTERP}
    assert (m == art.MASK_TRACED).sum() == st["rays_traced"] == sum(st["rays_per_level"])
    rng = np.random.default_rng(42)
    traced = np.flatnonzero(m.ravel() == art.MASK_TRACED)
    pick = rng.choice(traced, size=256, replace=False)
    ref, info = O.trace_pixels(O.make_job(**params), pick.astype(np.int64))
    got = g.ravel()[pick]
    if precision == "fp64":
        assert _close(got, ref[:, 0]).sum() == 0
    else:
        mse = np.sum((got - ref[:, 0]) ** 2) / (got.size * np.mean(ref[:, 0]) ** 2)
        assert mse < 1e-5, mse
    interp = np.flatnonzero(m.ravel() == art.MASK_INTERP)
    for p in rng.choice(interp, size=2000, replace=False):
        j, i = divmod(int(p), nx)
        k, s = _level_of(i, j, params["levels"])
        oi, oj = (i // s) % 2, (j // s) % 2
        if oi and oj:
            ref_v = 0.25 * (((g[j - s, i - s] + g[j + s, i - s]) + g[j - s, i + s]) + g[j + s, i + s])
        elif oi:
            ref_v = 0.5 * (g[j, i - s] + g[j, i + s])
        else:
            ref_v = 0.5 * (g[j - s, i] + g[j + s, i])
        assert g[j, i] == ref_v
    if precision != "fp64":
        assert 0 < st["rays_fp64"] < 0.2 * st["rays_traced"]
