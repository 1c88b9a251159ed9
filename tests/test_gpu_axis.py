"""Adaptive sampling along a third axis (frequency or time; the Sec. 6 proposal) on the GPU
(art_render_axis) against the oracle (oracle/axis.py): on a precomputed cube the decisions and
interpolants must be identical; with tracing (frequencies of the thermal-synchrotron disk) the
values must match the FP64 oracle per pixel."""
import numpy as np
import pytest

import oracle as O
from oracle import axis as A
from paper_2103_07417_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("F,levels3,R", [(17, 4, 2e-3), (9, 2, 1e-2), (13, 2, 0.0)])
def test_axis_logic_on_a_cube_matches_oracle(ctx, F, levels3, R):
    from paper_2103_07417_gb300 import art
    # 41 x 33 images with two planes (subring planes of an unpolarized job)
    job = art.make_job(**W.schwarzschild_129(n0x=6, n0y=5, levels=3, subrings=2))
    rng = np.random.default_rng(F)
    f = np.arange(F)[:, None, None, None]
    base = W.smooth_image(2, 41, 33)[None, None]
    cube = base * (1.0 + 0.3 * np.sin(0.4 * f + rng.uniform(0, 6, (1, 2, 33, 41)))) \
        + 0.02 * rng.uniform(size=(F, 2, 33, 41))
    truth = [torch.from_numpy(np.ascontiguousarray(cube[k])).cuda() for k in range(F)]
    imgs = [torch.empty_like(t) for t in truth]
    amask = torch.zeros((F, 33, 41), dtype=torch.uint8, device="cuda")
    st = ctx.art_render_axis([job] * F, levels3, R, R, imgs, amask=amask, truth=truth)
    ref, rmask, counts, _ = A.render_axis(F, levels3, R, R, truth=cube)
    np.testing.assert_array_equal(amask.cpu().numpy(), rmask)
    got = np.stack([t.cpu().numpy() for t in imgs])
    np.testing.assert_array_equal(got, ref)
    assert [s["rays_traced"] for s in st] == counts
    assert 0 < sum(counts[1:-1]) < (F - 1) * 33 * 41 or R == 0.0


def test_axis_frequencies_of_the_disk_match_oracle(ctx):
    """The thermal-synchrotron disk at 9 frequencies from 115 to 460 GHz (3 base frequencies,
    2 axis levels), 33^2 images (17^2 base, 1 spatial level), FP64, the axis combined with the
    spatial scheme: base images, traced, spatially and axially interpolated points against the
    oracle; masks agree except where an estimate sits at a tolerance (the two tracers agree to
    ~1e-7 relative, not bit for bit); fewer rays than independent renders of every frequency."""
    from paper_2103_07417_gb300 import art
    F, L3, R = 9, 2, 3e-3
    nus = 230e9 * 2.0 ** ((np.arange(F) - 4) / 4.0)
    params = [W.kerr_disk_2049(n0x=17, n0y=17, levels=1, stokes=1, precision="fp64",
                               crit_band=0.0, nu_hz=float(nu), R_rel=R, R_abs=R) for nu in nus]
    jobs = [art.make_job(**p) for p in params]
    nx, ny = art.art_image_size(jobs[0])
    imgs = [torch.empty((1, ny, nx), dtype=torch.float64, device="cuda") for _ in range(F)]
    amask = torch.zeros((F, ny, nx), dtype=torch.uint8, device="cuda")
    st = ctx.art_render_axis(jobs, L3, R, R, imgs, amask=amask)
    ref, rmask, counts, norm = A.render_axis_jobs([O.make_job(**p) for p in params], L3, R, R)
    gm = amask.cpu().numpy()
    got = np.stack([t.cpu().numpy() for t in imgs])
    diff = gm != rmask
    print("axis mask differences", int(diff.sum()), "rays", [x["rays_traced"] for x in st], counts)
    assert diff.mean() < 2e-3
    same = np.broadcast_to(~diff[:, None], got.shape)
    peak = np.abs(ref).max()
    scale = np.maximum(np.abs(ref), 1e-6 * peak)
    assert (np.abs(got - ref)[same] <= 1e-6 * scale[same]).all()
    assert [x["rays_traced"] for x in st] == counts or diff.any()
    # every sample rendered on its own traces at least as many rays
    solo = sum(ctx.render(j)[2]["rays_traced"] for j in jobs)
    assert sum(x["rays_traced"] for x in st) < solo
    assert (gm == art.MASK_AXIS).any()
