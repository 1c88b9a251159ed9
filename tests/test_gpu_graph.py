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
    ("cfg1_polarized", W.cfg1(n0x=65, n0y=65, levels=3)),
    ("cfg2_grid", W.cfg2(n0x=65, n0y=57, levels=3)),
    ("cfg0_fp64", W.cfg0(precision="fp64")),
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
    a = art.make_job(**W.cfg1(n0x=33, n0y=33, levels=2))
    b = art.make_job(**W.cfg1(n0x=33, n0y=33, levels=2, incl_deg=60.0))
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
    job = art.make_job(**W.cfg1(n0x=33, n0y=33, levels=2, proposal=1))
    img = torch.empty((4, 129, 129), dtype=torch.float64, device="cuda")
    mask = torch.empty((129, 129), dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="unsupported"):
        ctx.art_graph_render(job, img, mask)
