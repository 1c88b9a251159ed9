"""Exact refinement decisions (ART_MIXED_EXACT) against the FP64 render, and the mixed modes'
hand-over of rays near a discontinuity of the emission model.

The mixed modes trace in FP32, whose intensities differ from FP64 by rounding amplified along the
ray (~1e-5 relative typically, up to ~1e-3 on lensed rays).  The refinement criterion of Sec. 3.2
compares estimates built from second differences of those values with the tolerances, so a point
whose estimate sits near a tolerance can be traced in one precision and interpolated in the other
(a "mask flip"), and on a coarse base a flip re-routes a whole subtree of later levels.  With exact
decisions every point whose estimate lies within the band of a tolerance is decided in FP64 on
exact stencil values (FP64 re-traces and recomputed interpolants), and the base level is FP64, so
the decisions are those of the FP64 render wherever the FP32 values place a point on the same side
of the band's edges as the FP64 values do.

Error measure (the mixed path's bound): sum over the image of (dI)^2 / (N Ibar^2) per plane, Ibar
the mean total intensity of the FP64 render (every Stokes plane and subring plane is measured
against the same Ibar)."""
import numpy as np
import pytest

import oracle as O
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
    yield c
    c.close()


def _bj(img, ref, stokes, subrings):
    """Per-plane sum (dI)^2 / (N Ibar^2), Ibar the mean total intensity of the reference."""
    planes = img.shape[0]
    tot = sum(ref[n * stokes] for n in range(max(subrings, 1)))
    ib = float(tot.double().mean())
    n = img[0].numel()
    return [float(((img[c] - ref[c]).double() ** 2).sum()) / (n * ib * ib) for c in range(planes)]


def _flip_distances(params, ref_plane, mask_ref, mask, norm):
    """For every point whose mask differs: the relative distance of the FP64 render's decision from
    flipping, from the oracle's estimates (Eqs. epabs, eprel) on the FP64 image's level lattice."""
    N = params["levels"]
    m0, m1 = mask_ref.cpu().numpy(), mask.cpu().numpy()
    jj, ii = np.nonzero(m0 != m1)
    if jj.size == 0:
        return []
    img = ref_plane.cpu().numpy()
    out = []
    for i, j in zip(ii, jj):
        k = N
        while k > 0 and i % (1 << (N - k + 1)) == 0 and j % (1 << (N - k + 1)) == 0:
            k -= 1
        s = 1 << (N - k)
        L = np.ascontiguousarray(img[::s, ::s])
        ny, nx = L.shape
        job = O.make_job(**W.job(n0x=(nx - 1) // 2 + 1, n0y=(ny - 1) // 2 + 1, levels=1,
                                 R_abs=params["R_abs"], R_rel=params["R_rel"],
                                 interp=params.get("interp", "linear"),
                                 edge_mode=params.get("edge_mode", "onesided")))
        m = np.zeros(L.shape, np.uint8)
        m[::2, ::2] = O.MASK_TRACED
        _, _, ea, er = O.refine_level(job, L, m, 1, norm)
        a, r = ea[j // s, i // s] / params["R_abs"] - 1.0, er[j // s, i // s] / params["R_rel"] - 1.0
        trace = a > 0 and r > 0
        out.append(min(a, r) if trace else (max(-a, -r) if (a <= 0 and r <= 0) else (-a if a <= 0 else -r)))
    return out


CASES = [
    ("schwarzschild_129", W.schwarzschild_129()),
    ("kerr_analytic_513", W.kerr_analytic_2049(n0x=33, n0y=33, levels=4)),
    ("kerr_disk_polarized_513", W.kerr_disk_2049(n0x=33, n0y=33, levels=4)),
    ("grmhd_1025", W.grmhd_8193(n0x=65, n0y=65, levels=4)),
    ("grmhd_nearest_513", W.grmhd_8193(n0x=33, n0y=33, levels=4, interp="nearest")),
    ("grmhd_edge_trace_513", W.grmhd_8193(n0x=33, n0y=33, levels=4, edge_mode="trace", crit_band=0.0)),
]


@pytest.mark.parametrize("name,params", CASES, ids=[c[0] for c in CASES])
def test_exact_decisions_small(ctx, name, params):
    """Masks equal the FP64 render's; every plane within the mixed bound; the closure ran."""
    from paper_2103_07417_gb300 import art
    ref, mref, sref = ctx.render(art.make_job(**{**params, "precision": "fp64"}))
    img, mask, st = ctx.render(art.make_job(**{**params, "precision": "mixed_exact"}))
    torch.cuda.synchronize()
    assert st["norm"] == sref["norm"]  # the base level is traced in FP64: bit-identical
    assert st["border_overflow"] == 0
    flips = int((mask != mref).sum())
    d = _flip_distances(params, ref[0], mref, mask, sref["norm"])
    assert all(x <= 1e-9 for x in d), (flips, d)
    assert max(_bj(img, ref, params.get("stokes", 1), params.get("subrings", 0))) <= 1e-5
    assert st["rays_per_level"] == sref["rays_per_level"]


@pytest.mark.parametrize("name", ["kerr_disk_2049", "grmhd_8193"])
def test_exact_decisions_full_size(ctx, name):
    """The 2049^2 polarized and 8193^2 grid workloads: masks equal the FP64 render's except where
    the FP64 estimate is within 1e-9 of a tolerance, and every plane (I, Q, U, V) within the
    mixed bound."""
    from paper_2103_07417_gb300 import art
    params = W.BENCH_WORKLOADS[name][1]()
    ref, mref, sref = ctx.render(art.make_job(**{**params, "precision": "fp64"}))
    img, mask, st = ctx.render(art.make_job(**{**params, "precision": "mixed_exact"}))
    torch.cuda.synchronize()
    d = _flip_distances(params, ref[0], mref, mask, sref["norm"])
    bj = _bj(img, ref, params.get("stokes", 1), params.get("subrings", 0))
    print(name, "flips", len(d), d[:8], "bj", bj, "exact rays", st["rays_exact"],
          "border", st["border_points"])
    assert st["border_overflow"] == 0
    assert all(x <= 1e-9 for x in d), d
    assert max(bj) <= 1e-5, bj


def test_exact_decisions_batch_images(ctx):
    """Every image of the 256-image mixed-parameter batch (subring planes n = 0, 1, 2) rendered
    with exact decisions (art_render_batch runs the images concurrently) against the FP64 batch: each
    plane of each image within the mixed bound, masks equal except within 1e-9 of a tolerance."""
    from paper_2103_07417_gb300 import art
    bp = W.grmhd_batch(seed=0, n=256)
    jx = [art.make_job(**{**p, "precision": "mixed_exact"}) for p in bp]
    j64 = [art.make_job(**{**p, "precision": "fp64"}) for p in bp]
    ix, mx, sx = ctx.render_batch(jx)
    i64, m64, s64 = ctx.render_batch(j64)
    torch.cuda.synchronize()
    worst, nflip = 0.0, 0
    for p, a, b, ma, mb, s in zip(bp, ix, i64, mx, m64, s64):
        worst = max(worst, max(_bj(a, b, 1, 3)))
        if not torch.equal(ma, mb):
            d = _flip_distances(p, b[0], mb, ma, s["norm"])  # the criterion reads plane 0
            nflip += len(d)
            assert all(x <= 1e-9 for x in d), d
    print("batch worst bj", worst, "flips", nflip)
    assert worst <= 1e-5


def test_exact_batch_equals_single_renders(ctx):
    """art_render_batch with exact decisions runs the single-image level loop of each image on
    sub-contexts with streams of their own, concurrently: images, masks and statistics equal the
    images rendered one at a time by art_render, bit for bit, in any batch order and size (a
    batch larger than the number of sub-contexts, images of different sizes and depths)."""
    from paper_2103_07417_gb300 import art
    bp = W.grmhd_batch(seed=4, n=40)
    jx = [art.make_job(**{**p, "precision": "mixed_exact"}) for p in bp]
    ix, mx, sx = ctx.render_batch(jx)
    torch.cuda.synchronize()
    for j, a, ma, sa in zip(jx, ix, mx, sx):
        b, mb, sb = ctx.render(j)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert torch.equal(ma, mb)
        for k in ("rays_per_level", "rays_exact", "border_points", "steps", "norm",
                  "kernel_launches"):
            assert sa[k] == sb[k], (k, sa[k], sb[k])


def test_mixed_hands_over_rays_near_emission_edges(ctx):
    """Mixed modes: a ray with a sample within rounding of the disk's inner edge is re-traced at
    high precision, so no FP32-traced intensity of the 2049^2 disk workload differs from the FP64
    trace of the same ray by more than FP32 rounding amplified along the ray (before the
    hand-over, rays grazing the edge differed by up to 110 %)."""
    from paper_2103_07417_gb300 import art
    params = W.kerr_disk_2049()
    j64 = art.make_job(**{**params, "precision": "fp64"})
    ref, mref, sref = ctx.render(j64)
    pix = torch.nonzero(mref.reshape(-1) == art.MASK_TRACED).reshape(-1).to(torch.int32)
    a, _ = ctx.trace_pixels(art.make_job(**params), pix)
    b, _ = ctx.trace_pixels(j64, pix)
    torch.cuda.synchronize()
    rel = ((a[:, 0] - b[:, 0]).abs() / (b[:, 0].abs() + 1e-3 * sref["norm"])).max().item()
    assert rel < 1e-2, rel
