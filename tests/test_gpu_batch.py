"""Batched rendering (art_render_batch): many images of different spins, inclinations, fields of
view, grids and depths in one pass per level must reproduce the images the single-image path
renders one at a time: identical masks and ray counts, and pixel values equal to rounding (the two
kernels compile the same per-ray arithmetic, but the compiler may fuse multiply-adds differently
when the job comes from a table in memory instead of a kernel parameter)."""
import numpy as np
import pytest

from paper_2103_07417_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snap():
    return W.grmhd_snapshot(seed=0)


@pytest.mark.parametrize("precision,stokes,model", [
    ("mixed_df", 1, "grid"), ("fp64", 1, "grid"), ("mixed", 4, "grid"), ("mixed_df", 1, "disk")])
def test_batch_equals_single_renders(snap, precision, stokes, model):
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    ctx.load_grid(snap)
    params = W.grmhd_batch(seed=3, n=7)
    if model == "disk":   # the thermal-synchrotron disk instead of the snapshot
        params = [W.kerr_disk_2049(a=p["a"], incl_deg=p["incl_deg"], fov=p["fov"], r_in=W.r_isco(p["a"]))
                  for p in params]
    elif stokes == 4:
        # at the workload's density the torus is Faraday thick (~1e3 rad), where the last-bit
        # differences between the two kernels' FP32 code grow into O(1) changes of Q and U; a
        # 100x lower mass unit keeps the rotation of order one
        for p in params:
            p["m_unit"] = 3e24
    for i, p in enumerate(params):       # keep the images small, levels 0 .. 4 mixed
        k = 5 + (i % 2)
        N = [0, 1, 2, 3, 4, 2, 3][i]
        p.update(n0x=(1 << (k - min(N, k - 2))) + 1, levels=min(N, k - 2), precision=precision,
                 stokes=stokes, subrings=3 if stokes == 1 else 1)
        p["n0y"] = p["n0x"] - 4 * (i % 3 == 0)
    jobs = [art.make_job(**p) for p in params]
    imgs, masks, stats = ctx.render_batch(jobs)
    for j, img, mask, st in zip(jobs, imgs, masks, stats):
        ref, ref_mask, ref_st = ctx.render(j)
        torch.cuda.synchronize()
        assert torch.equal(mask, ref_mask)
        g, r = img.cpu().numpy(), ref.cpu().numpy()
        if stokes == 4:   # Q, U, V on the scale of the pixel's I
            scale = np.maximum(np.abs(r[0]), 1e-6 * np.abs(r[0]).max())[None]
        else:
            scale = np.maximum(np.abs(r), 1e-6 * np.abs(r).max())
        rel = np.max(np.abs(g - r) / scale)
        # The two renders run different kernels (the batched one reads each ray's job from a table;
        # the single-image FP32 and double-float passes may split each step over a pair of warps):
        # in FP64 the analytic models agree to ~1e-13 and the grid model's longer chains (exp of
        # arguments ~ -60) to a few ulps more.  In the FP32 pass the last-bit differences are FP32
        # rounding (~1e-7 of I) and can also move a ray whose swept angle sits at the re-trace
        # threshold from one precision to the other, a change of the size of the FP32 error
        # itself (~1e-4 of I, inside the 1e-5 MSE bound).  So the paths with an FP32 pass are held
        # to: 1e-3 of the pixel's I except on at most 1 % of the pixels (a moved ray and the
        # pixels interpolated from it), and an MSE between the two (all Stokes planes, relative to
        # the mean intensity squared) 10x below the mixed path's 1e-5 bound.
        if precision != "fp64":
            tol = 1e-3
            moved = np.abs(g - r) > tol * scale
            assert moved.mean() <= 1e-2, moved.mean()
            assert np.mean((g - r) ** 2) / np.mean(r[0]) ** 2 < 1e-6
        else:
            tol = 1e-12 if model == "disk" else 1e-10
            assert rel <= tol, rel
        assert st["rays_per_level"] == ref_st["rays_per_level"]
        # the normalisation is a statistic of the traced intensities: the same bound
        assert st["norm"] == pytest.approx(ref_st["norm"], rel=max(tol, 1e-13))
    ctx.close()


def test_batch_rejects_mixed_kinds():
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    a = art.make_job(**W.schwarzschild_129(n0x=9, n0y=9, levels=1))
    b = art.make_job(**W.schwarzschild_129(n0x=9, n0y=9, levels=1, precision="mixed"))
    with pytest.raises(RuntimeError):
        ctx.render_batch([a, b])
    ctx.close()


def _small_batch(seed, n, band):
    """A mixed-parameter batch of small images (65^2 and 129^2, 2-4 levels) with the given
    near-critical band width on every image (or a list of widths, one per image)."""
    params = W.grmhd_batch(seed=seed, n=n)
    bands = band if isinstance(band, list) else [band] * n
    for i, p in enumerate(params):
        k = 6 + (i % 2)
        N = 2 + (i % 3)
        p.update(n0x=(1 << (k - N)) + 1, n0y=(1 << (k - N)) + 1, levels=N, crit_band=bands[i])
    return params


@pytest.mark.parametrize("band", [0.03, 0.5, "mixed"])
def test_batch_band_equals_plain_batch(snap, band):
    """The near-critical band in the batched path: every image and mask equals the batch rendered
    without it bit for bit, with the same rays per level; speculative rays were traced."""
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    ctx.load_grid(snap)
    n = 12
    widths = [0.03 if i % 2 else 0.0 for i in range(n)] if band == "mixed" else band
    plain = [art.make_job(**p) for p in _small_batch(11, n, 0.0)]
    banded = [art.make_job(**p) for p in _small_batch(11, n, widths)]
    i0, m0, s0 = ctx.render_batch(plain)
    i1, m1, s1 = ctx.render_batch(banded)
    torch.cuda.synchronize()
    for a, b in zip(i0, i1):
        assert torch.equal(a, b)
    for a, b in zip(m0, m1):
        assert torch.equal(a, b)
    for a, b in zip(s0, s1):
        assert a["rays_per_level"] == b["rays_per_level"]
    assert s0[0]["rays_speculative"] == 0
    assert 0 < s1[0]["rays_spec_used"] <= s1[0]["rays_speculative"]
    assert s1[0]["rays_fp64"] >= s0[0]["rays_fp64"]
    ctx.close()


def test_batch_band_without_masks(snap):
    """Images whose caller passes no mask speculate on context-owned scratch masks: the images
    equal those rendered with masks."""
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    ctx.load_grid(snap)
    jobs = [art.make_job(**p) for p in _small_batch(12, 6, 0.03)]
    imgs, masks, _ = ctx.render_batch(jobs)
    bare = [torch.full_like(t, float("nan")) for t in imgs]
    ctx.art_render_batch(jobs, bare, None, stats=False)
    torch.cuda.synchronize()
    for a, b in zip(imgs, bare):
        assert torch.equal(a, b)
    ctx.close()


def test_batch_band_moves_retraces_to_the_base_pass(snap):
    """With the band, the double-float passes after the base level of a mixed-parameter batch
    re-trace (almost) nothing: the photon-ring rays of every level of every image were traced
    with the base level.  No magnetisation cut and no subring planes here (sigma_cut 1e30,
    subrings 0), so no ray is handed over for a sample near the cut or a marginal polar turn,
    which can happen at any level."""
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    ctx.load_grid(snap)
    jobs = [art.make_job(**p) for p in W.grmhd_batch(seed=0, n=32, sigma_cut=1e30, subrings=0)]
    imgs, masks, st = ctx.render_batch(jobs)
    ctx.art_profile(True)
    ctx.art_render_batch(jobs, imgs, masks, stats=False)
    recs = ctx.art_profile_read()
    ctx.art_profile(False)
    df = [r for r in recs if r["kind"] == "trace_df"]
    later = sum(r["steps"] for r in df if r["level"] > 0)
    print("df steps per level", [(r["level"], r["steps"]) for r in df])
    assert df[0]["level"] == 0 and df[0]["steps"] > 0
    assert later <= 0.05 * df[0]["steps"], [(r["level"], r["steps"]) for r in df]
    ctx.close()
