"""The learned path of the render (speculative tracing of blocks the network proposes, the exact
criterion still deciding every point), its training samples, and what the trained network gains.

Invariant: a learned render equals the plain render of the same job bit for bit (image, mask,
rays per level); only the time at which rays are traced changes."""
import numpy as np
import pytest

from paper_2103_07417_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snap():
    return W.grmhd_snapshot(seed=0)


@pytest.fixture(scope="module")
def ctx(snap):
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    c.load_grid(snap)
    c.art_cnn_load(W.cnn_init(7))
    yield c
    c.close()


CASES = [
    ("grmhd_8193", W.grmhd_8193(n0x=33, n0y=33, levels=4, fov=60.0, crit_band=0.0)),
    ("kerr_disk_unpolarized", W.kerr_disk_2049(n0x=17, n0y=17, levels=4, stokes=1, crit_band=0.0)),
    ("kerr_disk_polarized_ragged", W.kerr_disk_2049(n0x=17, n0y=13, levels=3, crit_band=0.0)),
    ("schwarzschild_fp64", W.schwarzschild_129(precision="fp64", n0x=17, n0y=17, levels=3)),
    ("kerr_disk_with_band", W.kerr_disk_2049(n0x=17, n0y=17, levels=4, stokes=1)),
]


@pytest.mark.parametrize("thr,depth", [(0.0, 1), (0.0, 3), (0.5, 2), (1.0, 2)])
@pytest.mark.parametrize("name,params", CASES, ids=[c[0] for c in CASES])
def test_learned_render_equals_plain(ctx, name, params, thr, depth):
    from paper_2103_07417_gb300 import art
    plain = art.make_job(**params)
    learned = art.make_job(**{**params, "proposal": 1, "proposal_p": thr, "proposal_depth": depth})
    img0, mask0, st0 = ctx.render(plain)
    img1, mask1, st1 = ctx.render(learned)
    torch.cuda.synchronize()
    assert torch.equal(mask0, mask1)
    assert torch.equal(img0, img1)
    assert st0["rays_per_level"] == st1["rays_per_level"]
    assert st1["rays_spec_used"] <= st1["rays_speculative"]
    if thr == 0.0:
        assert st1["rays_speculative"] > 0 and st1["rays_spec_used"] > 0
    if thr == 1.0 and params.get("crit_band", 0.0) == 0.0:
        assert st1["rays_speculative"] == 0
    assert int(((mask1 == 1) | (mask1 == 2)).sum()) == mask1.numel()


def test_training_sample_matches_host_definition(ctx):
    """Features of a level lattice: asinh(I / (R_abs I_norm)) from the image and the render's
    normalisation, and at traced points 3 / max(r_min, 1) and the polar turns of the ray;
    targets: any point of level L + 2 or L + 3 traced in the 4 x 4-cell block."""
    from paper_2103_07417_gb300 import art
    p = W.kerr_disk_2049(n0x=17, n0y=17, levels=4, stokes=1)
    job = art.make_job(**p)
    img, mask, st = ctx.render(job)
    L = 1
    feat, tgt = ctx.art_cnn_sample(job, img[0], mask, L)
    f, t = feat.cpu().numpy(), tgt.cpu().numpy()
    I, m = img[0].cpu().numpy(), mask.cpu().numpy()
    s = 1 << (p["levels"] - L)
    np.testing.assert_allclose(f[..., 0], np.arcsinh(I[::s, ::s] / (p["R_abs"] * st["norm"])),
                               rtol=1e-5, atol=1e-6)
    # the base level (traced everywhere) against the tracer's own diagnostics
    s0 = 1 << p["levels"]
    nx = m.shape[1]
    jj, ii = np.mgrid[0:m.shape[0]:s0, 0:nx:s0]
    pix = (jj * nx + ii).ravel().astype(np.int32)
    _, aux = ctx.trace_pixels(job, torch.from_numpy(pix).cuda())
    fr = f[::s0 // s, ::s0 // s].reshape(-1, 3)
    np.testing.assert_allclose(fr[:, 1], 3.0 / np.maximum(aux["min_r"].cpu().numpy(), 1.0), rtol=1e-6)
    np.testing.assert_array_equal(fr[:, 2], aux["nturn"].cpu().numpy().astype(np.float32))
    ny_, nx_ = m.shape
    H4, W4 = t.shape
    half = s // 2
    st_ = max(s // 8, 1)
    yy, xx = np.mgrid[0:ny_, 0:nx_]
    deep = ((xx % half != 0) | (yy % half != 0)) & (xx % st_ == 0) & (yy % st_ == 0)
    for hy in range(H4):
        for hx in range(W4):
            blk = (slice(hy * 4 * s, (hy + 1) * 4 * s), slice(hx * 4 * s, (hx + 1) * 4 * s))
            want = bool(((m[blk] == 1) & deep[blk]).any())
            assert t[hy, hx] == float(want), (hy, hx)


def test_trained_proposal_gain(snap):
    """Train on 96 seeded plain renders (the library's tensor-core forward/backward and Adam),
    then: on 9 held-out jobs the network finds the refined blocks (at p > 0.1 recall >= 0.95 with
    precision >= 1.3x the base rate, and a precision >= 2x the base rate at 80 % recall), and on the
    2049^2 analytic-emissivity workload the learned render (lookahead 3 levels, the best of
    p > 0.3, 0.5, 0.7) is at least 1.2x faster than the plain one (median of 5 CUDA-event timed
    renders each), with image and mask unchanged.  Both renders leave the near-critical band
    speculation off, so the gain is the network's own."""
    from paper_2103_07417_gb300 import art, learn
    ctx, hist = learn.trained_context(seed=0, n_jobs=96, epochs=12, snapshot=snap)
    try:
        assert hist[-1] < 0.6 * hist[0], hist
        held = learn.training_jobs(123, 9)
        hs = learn.collect(ctx, held)
        lo = learn.block_scores(ctx, hs, 0.1)
        base = lo["positives"] / sum(t.numel() for _, t in hs)
        # training is reproducible (fixed-order gradient sums); the bounds below keep a margin
        # under the precisions this training reaches (printed with -s)
        print("held-out blocks at p > 0.1:", lo, "base rate", base)
        assert lo["recall"] >= 0.95 and lo["precision"] >= 1.3 * base, (lo, base)
        # precision at 80 % recall: the best precision over thresholds whose recall is >= 0.8
        sweep = [learn.block_scores(ctx, hs, thr) for thr in (0.15, 0.2, 0.25, 0.3, 0.35, 0.4)]
        p80 = max([sc["precision"] for sc in sweep if sc["recall"] >= 0.8], default=0.0)
        print("precision at 80 % recall:", p80, "sweep", sweep)
        assert p80 >= 2.0 * base, (sweep, base)
        p = W.kerr_analytic_2049(crit_band=0.0)
        plain = art.make_job(**p)
        # the threshold is a setting of the render: the best of three (a lower one proposes more
        # blocks than the exact criterion refines, a higher one fewer)
        lrns = [art.make_job(**{**p, "proposal": 1, "proposal_p": thr, "proposal_depth": 3})
                for thr in (0.3, 0.5, 0.7)]
        img0, mask0, st0 = ctx.render(plain)
        for lrn in lrns:
            img1, mask1, st1 = ctx.render(lrn)
            assert torch.equal(img0, img1) and torch.equal(mask0, mask1)

        def med(job):
            ts = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                ctx.art_render(job, img0, mask0, stats=False)
                e1.record(ctx.stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return float(np.median(ts))

        t_plain, t_learned = med(plain), min(med(lrn) for lrn in lrns)
        assert t_learned * 1.2 <= t_plain, (t_plain, t_learned)
    finally:
        ctx.close()


def test_training_is_reproducible(snap):
    """The gradient kernels reduce their per-CTA partial sums in a fixed order (no floating-point
    atomics), so two trainings from the same initial network on the same renders end with the
    same parameters bit for bit."""
    from paper_2103_07417_gb300 import learn
    outs = []
    for _ in range(2):
        ctx, hist = learn.trained_context(seed=1, n_jobs=4, epochs=2, snapshot=snap)
        try:
            outs.append((ctx.art_cnn_read(), list(hist)))
        finally:
            ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
