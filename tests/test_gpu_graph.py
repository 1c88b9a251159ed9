"""art_graph_render: the level loop captured once into a CUDA graph and replayed gives the
images and masks of art_render, bit for bit, on consecutive calls and after a change of job
(which captures again); learned jobs are refused."""
import numpy as np
import pytest
import torch

from paper_2103_07417_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    c.load_grid(W.grmhd_snapshot(seed=0))
    yield c
    c.close()


CASES = [
    ("kerr_disk_polarized", W.kerr_disk_2049(n0x=65, n0y=65, levels=3)),
    ("grmhd_grid", W.grmhd_8193(n0x=65, n0y=57, levels=3)),
    ("schwarzschild_fp64", W.schwarzschild_129(precision="fp64")),
]


@pytest.mark.parametrize("name,params", CASES, ids=[c[0] for c in CASES])
def test_graph_replay_equals_render(ctx, name, params):
    from paper_2103_07417_gb300 import art
    job = art.make_job(**params)
    ref_img, ref_mask, _ = ctx.render(job)
    img = torch.full_like(ref_img, np.nan)
    mask = torch.zeros_like(ref_mask)
    for _ in range(2):   # capture + replay, then replay
        img.fill_(np.nan)
        mask.zero_()
        ctx.art_graph_render(job, img, mask)
        torch.cuda.synchronize()
        assert torch.equal(img, ref_img) and torch.equal(mask, ref_mask)


def test_graph_recaptures_on_a_new_job(ctx):
    from paper_2103_07417_gb300 import art
    a = art.make_job(**W.kerr_disk_2049(n0x=33, n0y=33, levels=2))
    b = art.make_job(**W.kerr_disk_2049(n0x=33, n0y=33, levels=2, incl_deg=60.0))
    img, mask, _ = ctx.render(a)
    ref_b, ref_mask_b, _ = ctx.render(b)
    ref_a, ref_mask_a, _ = ctx.render(a)
    ctx.art_graph_render(a, img, mask)
    torch.cuda.synchronize()
    assert torch.equal(img, ref_a) and torch.equal(mask, ref_mask_a)
    ctx.art_graph_render(b, img, mask)
    torch.cuda.synchronize()
    assert torch.equal(img, ref_b) and torch.equal(mask, ref_mask_b)


def test_graph_refuses_learned_jobs(ctx):
    from paper_2103_07417_gb300 import art
    job = art.make_job(**W.kerr_disk_2049(n0x=33, n0y=33, levels=2, proposal=1))
    img = torch.empty((4, 129, 129), dtype=torch.float64, device="cuda")
    mask = torch.empty((129, 129), dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="unsupported"):
        ctx.art_graph_render(job, img, mask)


def test_graph_batch_replay_equals_batch_render(ctx):
    """A mixed-parameter batch (mixed sizes and levels) replayed from its graph: images and masks
    of art_render_batch, on two consecutive calls, and again after a larger single render made the
    context reallocate its ray queue (the graph is captured anew)."""
    from paper_2103_07417_gb300 import art
    params = W.grmhd_batch(seed=5, n=6)
    for i, p in enumerate(params):
        k = 5 + (i % 2)
        N = [1, 2, 3, 2, 3, 1][i]
        p.update(n0x=(1 << (k - N)) + 1, n0y=(1 << (k - N)) + 1, levels=N)
    jobs = [art.make_job(**p) for p in params]
    ref_imgs, ref_masks, _ = ctx.render_batch(jobs)
    imgs = [torch.full_like(t, np.nan) for t in ref_imgs]
    masks = [torch.zeros_like(m) for m in ref_masks]
    for rnd in range(3):
        if rnd == 2:   # a larger render grows the single-image scratch (and not the batch's)
            ctx.render(art.make_job(**W.kerr_disk_2049(n0x=129, n0y=129, levels=3)))
        for t in imgs:
            t.fill_(np.nan)
        for m in masks:
            m.zero_()
        ctx.art_graph_render_batch(jobs, imgs, masks)
        torch.cuda.synchronize()
        for a, b in zip(imgs, ref_imgs):
            assert torch.equal(a, b)
        for a, b in zip(masks, ref_masks):
            assert torch.equal(a, b)


def test_graph_single_recaptures_after_scratch_growth(ctx):
    """A replayed graph must not use buffers a later, larger render reallocated."""
    from paper_2103_07417_gb300 import art
    small = art.make_job(**W.kerr_disk_2049(n0x=33, n0y=33, levels=2))
    img, mask, _ = ctx.render(small)
    ref = img.clone()
    ctx.art_graph_render(small, img, mask)
    big = art.make_job(**W.kerr_disk_2049(n0x=257, n0y=257, levels=3))
    ctx.render(big)      # grows the ray queue
    img.fill_(np.nan)
    ctx.art_graph_render(small, img, mask)
    torch.cuda.synchronize()
    assert torch.equal(img, ref)


def test_graph_batch_without_masks(ctx):
    """A batch replayed without caller masks: the near-critical band keeps its state in
    context-owned scratch masks, bound before the capture; images equal the batch render's."""
    from paper_2103_07417_gb300 import art
    params = W.grmhd_batch(seed=8, n=5)
    for i, p in enumerate(params):
        N = 2 + (i % 2)
        p.update(n0x=(1 << (6 - N)) + 1, n0y=(1 << (6 - N)) + 1, levels=N, crit_band=0.03)
    jobs = [art.make_job(**p) for p in params]
    ref_imgs, _, _ = ctx.render_batch(jobs)
    imgs = [torch.full_like(t, np.nan) for t in ref_imgs]
    for _ in range(2):
        for t in imgs:
            t.fill_(np.nan)
        ctx.art_graph_render_batch(jobs, imgs, None)
        torch.cuda.synchronize()
        for a, b in zip(imgs, ref_imgs):
            assert torch.equal(a, b)
