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


@pytest.mark.parametrize("precision,stokes", [("mixed_df", 1), ("fp64", 1), ("mixed", 4)])
def test_batch_equals_single_renders(precision, stokes):
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    params = W.cfg3(seed=3, n=7)
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
        scale = np.maximum(np.abs(r), 1e-6 * np.abs(r).max())
        rel = np.max(np.abs(g - r) / scale)
        assert rel <= 1e-12, rel
        assert st["rays_per_level"] == ref_st["rays_per_level"]
        assert st["norm"] == pytest.approx(ref_st["norm"], rel=1e-13)
    ctx.close()


def test_batch_rejects_mixed_kinds():
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    a = art.make_job(**W.cfg0(n0x=9, n0y=9, levels=1))
    b = art.make_job(**W.cfg0(n0x=9, n0y=9, levels=1, precision="mixed"))
    with pytest.raises(RuntimeError):
        ctx.render_batch([a, b])
    ctx.close()
