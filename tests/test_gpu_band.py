"""Speculation of the near-critical band (pixels whose camera rays lie near the Kerr critical curve
are traced with the base level): images and masks equal the plain render's bit for bit, and on the
2049^2 polarized workload every high-precision re-trace happens in the base level's pass."""
import pytest

from paper_2103_07417_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    c.load_grid(W.grmhd_snapshot(seed=0))
    yield c
    c.close()


CASES = [
    ("kerr_disk_polarized", W.kerr_disk_2049(n0x=33, n0y=33, levels=3)),
    ("kerr_disk_retrograde_i75", W.kerr_disk_2049(a=-0.6, incl_deg=75.0, r_in=W.r_isco(-0.6), n0x=17, n0y=17,
                                   levels=3, stokes=1)),
    ("grmhd_grid", W.grmhd_8193(n0x=33, n0y=33, levels=4, fov=60.0)),
    ("schwarzschild_fp64", W.schwarzschild_129(precision="fp64", levels=3, n0x=17, n0y=17)),
    ("kerr_analytic_mixed", W.kerr_analytic_2049(n0x=33, n0y=33, levels=3)),
]


@pytest.mark.parametrize("band", [0.005, 0.03, 0.5])
@pytest.mark.parametrize("name,params", CASES, ids=[c[0] for c in CASES])
def test_band_render_equals_plain(ctx, name, params, band):
    from paper_2103_07417_gb300 import art
    img0, mask0, st0 = ctx.render(art.make_job(**{**params, "crit_band": 0.0}))
    img1, mask1, st1 = ctx.render(art.make_job(**{**params, "crit_band": band}))
    torch.cuda.synchronize()
    assert torch.equal(img0, img1) and torch.equal(mask0, mask1)
    assert st0["rays_per_level"] == st1["rays_per_level"]
    # re-traced rays include the speculative ones the criterion later discards
    assert st1["rays_fp64"] >= st0["rays_fp64"]
    assert st1["rays_spec_used"] <= st1["rays_speculative"]
    if band == 0.5 and params["levels"] > 0:
        assert st1["rays_speculative"] > 0


def test_band_moves_every_retrace_to_the_base_pass(ctx):
    """2049^2 polarized workload with the default band: the double-float passes of levels 1..4
    trace no ray (all near-critical rays of those levels were traced with level 0).  The disk
    here extends to the photon orbit (r_in = 0), so no ray is handed over for a sample near the
    inner edge, which can happen at any level."""
    from paper_2103_07417_gb300 import art
    job = art.make_job(**W.kerr_disk_2049(r_in=0.0))
    img, mask, st = ctx.render(job)
    ctx.art_profile(True)
    ctx.art_render(job, img, mask, stats=False)
    recs = ctx.art_profile_read()
    ctx.art_profile(False)
    df = [r for r in recs if r["kind"] == "trace_df"]
    assert len(df) == 5 and df[0]["steps"] > 0
    assert all(r["steps"] == 0 for r in df[1:]), [r["steps"] for r in df]
    assert st["rays_fp64"] > 1000
