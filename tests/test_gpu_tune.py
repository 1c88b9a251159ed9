"""Trace scheduling (art_set_tune / art_get_tune: FP32 kernel-form thresholds and the persistent
grids' blocks per SM) and the autotuner (art_autotune): the forms and grids give bit-identical rays,
so every setting renders the same image and mask, and the autotuner leaves one of its candidates in
the context."""
import numpy as np
import pytest
import torch

from paper_2103_07417_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    yield c
    c.close()


def test_tune_roundtrip_and_validation(ctx):
    from paper_2103_07417_gb300 import art
    assert ctx.art_get_tune() == art.TUNE_DEFAULT
    ctx.art_set_tune(16, 128, 1, 2, 64)
    assert ctx.art_get_tune() == (16, 128, 1, 2, 64)
    for bad in ((-1, 64), (64, 32), (0, 5000), (16, 128, -1, 0), (16, 128, 0, 65),
                (16, 128, 1, 0, -1), (16, 128, 1, 0, 5000)):
        with pytest.raises(RuntimeError):
            ctx.art_set_tune(*bad)
    assert ctx.art_get_tune() == (16, 128, 1, 2, 64)
    ctx.art_set_tune()
    assert ctx.art_get_tune() == art.TUNE_DEFAULT


@pytest.mark.parametrize("name,over", [
    ("kerr_disk_polarized", dict(n0x=65, n0y=65, levels=3)),
    ("kerr_analytic_2049", dict(n0x=65, n0y=49, levels=3)),
])
def test_every_setting_renders_the_same_image(ctx, name, over):
    """One-thread only, pair only, quad-heavy and pair-heavy settings: identical images, masks
    and ray counts (every level's FP32 launch changes form between them)."""
    from paper_2103_07417_gb300 import art
    p = (W.kerr_disk_2049 if name == "kerr_disk_polarized" else W.kerr_analytic_2049)(**over)
    job = art.make_job(**p)
    ref = None
    for q, pr, b64, b32 in ((0, 0, 0, 0), (0, 4096, 0, 0), (4096, 4096, 0, 0), (32, 64, 0, 0),
                            (8, 16, 0, 0), (32, 64, 1, 1), (0, 0, 2, 1), (4096, 4096, 1, 2)):
        ctx.art_set_tune(q, pr, b64, b32)
        img, mask, st = ctx.render(job)
        if ref is None:
            ref = (img.clone(), mask.clone(), st["rays_per_level"])
        else:
            assert torch.equal(img, ref[0]) and torch.equal(mask, ref[1]), (q, pr, b64, b32)
            assert st["rays_per_level"] == ref[2]
    ctx.art_set_tune()


def test_autotune_keeps_a_candidate_and_the_image(ctx):
    from paper_2103_07417_gb300 import art
    job = art.make_job(**W.kerr_disk_2049(n0x=65, n0y=65, levels=3))
    img0, mask0, _ = ctx.render(job)
    img = torch.empty_like(img0)
    mask = torch.empty_like(mask0)
    best, ms = ctx.art_autotune(job, img, mask, reps=2)
    q, pr, b64, b32, q64 = best
    assert 0 <= q <= pr <= 4096 and ms > 0 and b64 in (0, 1, 2) and b32 in (0, 1, 2)
    assert q64 in (0, 32, 64)
    assert ctx.art_get_tune() == best
    assert torch.equal(img, img0) and torch.equal(mask, mask0)
    with pytest.raises(RuntimeError):
        ctx.art_autotune(job, img, mask, reps=0)
    assert ctx.art_get_tune() == best
    ctx.art_set_tune()


def test_fp64_grids_render_the_same_image():
    """Exact decisions (FP64 base level and closure passes) under every FP64 grid size and form
    (pair only, quad for short queues, quad for every queue): the same image, mask and rays."""
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    try:
        c.load_grid(W.grmhd_snapshot(seed=0))
        job = art.make_job(**W.grmhd_8193(n0x=33, n0y=33, levels=4, precision="mixed_exact"))
        ref = None
        for b64, q64 in ((0, 0), (1, 0), (2, 0), (3, 0), (0, 32), (1, 32), (3, 32), (1, 4096)):
            c.art_set_tune(32, 64, b64, 0, q64)
            img, mask, st = c.render(job)
            if ref is None:
                ref = (img.clone(), mask.clone(), st["rays_per_level"], st["rays_exact"])
            else:
                assert torch.equal(img, ref[0]) and torch.equal(mask, ref[1]), (b64, q64)
                assert (st["rays_per_level"], st["rays_exact"]) == ref[2:]
    finally:
        c.close()


@pytest.mark.parametrize("name", ["kerr_disk_polarized", "kerr_analytic"])
def test_fp64_forms_render_the_same_image(ctx, name):
    """FP64 renders (every level an FP64 launch) with the pair form only, the quad form for short
    queues and the quad form for every queue: identical images, masks and ray counts."""
    from paper_2103_07417_gb300 import art
    f = W.kerr_disk_2049 if name == "kerr_disk_polarized" else W.kerr_analytic_2049
    job = art.make_job(**f(n0x=33, n0y=33, levels=3, precision="fp64"))
    ref = None
    for b64, q64 in ((1, 0), (1, 32), (0, 4096), (2, 4096)):
        ctx.art_set_tune(32, 64, b64, 0, q64)
        img, mask, st = ctx.render(job)
        if ref is None:
            ref = (img.clone(), mask.clone(), st["rays_per_level"])
        else:
            assert torch.equal(img, ref[0]) and torch.equal(mask, ref[1]), (b64, q64)
            assert st["rays_per_level"] == ref[2]
    ctx.art_set_tune()
