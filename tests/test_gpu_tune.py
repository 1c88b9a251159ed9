"""Kernel-form thresholds (art_set_tune / art_get_tune) and the autotuner (art_autotune): the
forms give bit-identical rays, so every setting renders the same image and mask, and the
autotuner leaves one of its candidates in the context."""
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
    ctx.art_set_tune(16, 128)
    assert ctx.art_get_tune() == (16, 128)
    for bad in ((-1, 64), (64, 32), (0, 5000)):
        with pytest.raises(RuntimeError):
            ctx.art_set_tune(*bad)
    assert ctx.art_get_tune() == (16, 128)
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
    for q, pr in ((0, 0), (0, 4096), (4096, 4096), (32, 64), (8, 16)):
        ctx.art_set_tune(q, pr)
        img, mask, st = ctx.render(job)
        if ref is None:
            ref = (img.clone(), mask.clone(), st["rays_per_level"])
        else:
            assert torch.equal(img, ref[0]) and torch.equal(mask, ref[1]), (q, pr)
            assert st["rays_per_level"] == ref[2]
    ctx.art_set_tune()


def test_autotune_keeps_a_candidate_and_the_image(ctx):
    from paper_2103_07417_gb300 import art
    job = art.make_job(**W.kerr_disk_2049(n0x=65, n0y=65, levels=3))
    img0, mask0, _ = ctx.render(job)
    img = torch.empty_like(img0)
    mask = torch.empty_like(mask0)
    (q, pr), ms = ctx.art_autotune(job, img, mask, reps=2)
    assert 0 <= q <= pr <= 4096 and ms > 0
    assert ctx.art_get_tune() == (q, pr)
    assert torch.equal(img, img0) and torch.equal(mask, mask0)
    with pytest.raises(RuntimeError):
        ctx.art_autotune(job, img, mask, reps=0)
    assert ctx.art_get_tune() == (q, pr)
    ctx.art_set_tune()
