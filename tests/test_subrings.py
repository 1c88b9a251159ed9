"""Subring decomposition (Sec. 5.1): emission is split by the number n of polar turning points
between the camera and the emission point, so a thin disk's image separates into subrings.

Oracle pin: for a face-on Schwarzschild thin disk the n-th subring narrows by the Lyapunov factor
exp(-gamma) with gamma = pi per step in n (Sec. 5.1: w_n ~ w_0 exp(-gamma n)).  GPU parity: the
subring planes of the CUDA tracer match the oracle's."""
import numpy as np
import pytest

import oracle as O
from paper_2103_07417_gb300 import workloads as W


def test_lyapunov_narrowing_of_subrings_schwarzschild():
    """Face-on Schwarzschild thin disk, camera at 1e4 M: the subring bands approach the critical
    curve geometrically.  In the strong-deflection regime (n = 2 -> 3) the outer edge of the band,
    the image of a fixed source radius, moves in by the Lyapunov factor exp(-gamma), gamma = pi
    (Sec. 5.1: delta rho_n ~ rho_c exp(-gamma n)); the peak brightness of the subrings stays
    roughly constant (Sec. 5.1)."""
    r_obs = 1.0e4
    p = W.schwarzschild_129(a=0.0, incl_deg=0.1, disk_w=0.02, subrings=4, r_obs=r_obs, step_frac=0.02)
    job = O.make_job(**p)
    rho_c = r_obs * np.tan(np.arcsin(np.sqrt(27.0) * np.sqrt(1 - 2 / r_obs) / r_obs))  # Synge
    d = np.geomspace(1e-6, 1.5, 5000)
    out, info = O.trace_screen(job, rho_c + d, np.zeros_like(d))
    edge = {}
    for n in (1, 2, 3):
        prof = out[:, n]
        edge[n] = d[np.flatnonzero(prof > 1e-3 * prof.max())[-1]]
    assert edge[3] / edge[2] == pytest.approx(np.exp(-np.pi), rel=0.05)
    assert 0.5 * np.exp(-np.pi) < edge[2] / edge[1] < 1.5 * np.exp(-np.pi)
    peaks = [out[:, n].max() for n in (1, 2, 3)]
    assert max(peaks) / min(peaks) < 1.35


def _agm_k(m):
    """Complete elliptic integral K(m) = pi / (2 AGM(1, sqrt(1 - m))) (Gauss), m < 1."""
    x, y = 1.0, np.sqrt(1.0 - m)
    for _ in range(40):
        x, y = 0.5 * (x + y), np.sqrt(x * y)
    return np.pi / (2.0 * x)


def _lyapunov_face_on(a):
    """Lyapunov exponent of the photon orbit a face-on observer sees (lambda = 0), from the
    photon-shell expressions (Sec. 5.1): gamma = 4 r sqrt(chi) / sqrt(-u_- a^2) K(u_+/u_-),
    chi = 1 - Delta / (r (r - 1)^2), u_pm = D_th +- sqrt(D_th^2 + eta/a^2),
    D_th = (1 - (eta + lambda^2)/a^2) / 2, with r from lambda_c(r) = 0 on Bardeen's curve."""
    from scipy.optimize import brentq
    lam = lambda r: (r * r * (3 - r) - a * a * (r + 1)) / (a * (r - 1))
    r = brentq(lam, 2 * (1 + np.cos(2 / 3 * np.arccos(-a))), 2 * (1 + np.cos(2 / 3 * np.arccos(a))))
    eta = r ** 3 * (4 * a * a - r * (r - 3) ** 2) / (a * a * (r - 1) ** 2)
    chi = 1 - (r * r - 2 * r + a * a) / (r * (r - 1) ** 2)
    dth = 0.5 * (1 - eta / (a * a))
    up, um = dth + np.sqrt(dth ** 2 + eta / a ** 2), dth - np.sqrt(dth ** 2 + eta / a ** 2)
    return 4 * r * np.sqrt(chi) / np.sqrt(-um * a * a) * _agm_k(up / um)


def test_lyapunov_narrowing_of_subrings_kerr():
    """Face-on Kerr disk (a = 0.94), camera at 1e4 M: from n = 2 to n = 3 the outer edge of the
    subring band moves towards the critical curve by exp(-gamma) with the Kerr exponent of the
    lambda = 0 photon orbit (gamma = 2.567, against pi for a = 0, to which the same expression
    tends).  The critical radius on the screen is found by bisection on capture."""
    assert _lyapunov_face_on(1e-3) == pytest.approx(np.pi, rel=1e-3)
    a = 0.94
    gamma = _lyapunov_face_on(a)
    assert gamma == pytest.approx(2.567, abs=2e-3)
    r_obs = 1.0e4
    p = W.schwarzschild_129(a=a, incl_deg=0.1, disk_w=0.02, subrings=4, r_obs=r_obs, step_frac=0.02)
    job = O.make_job(**p)
    lo, hi = 4.0, 6.0
    for _ in range(45):
        mid = 0.5 * (lo + hi)
        _, info = O.trace_screen(job, [mid], [0.0])
        if info["status"][0] == O.RAY_CAPTURED:
            lo = mid
        else:
            hi = mid
    rho_c = hi
    d = np.geomspace(1e-6, 1.5, 3000)
    out, info = O.trace_screen(job, rho_c + d, np.zeros_like(d))
    edge = {n: d[np.flatnonzero(out[:, n] > 1e-3 * out[:, n].max())[-1]] for n in (1, 2, 3)}
    assert edge[3] / edge[2] == pytest.approx(np.exp(-gamma), rel=0.05)
    assert 0.5 * np.exp(-gamma) < edge[2] / edge[1] < 1.5 * np.exp(-gamma)


def test_subring_planes_sum_to_total():
    p = W.schwarzschild_129(a=0.94, incl_deg=17.0, disk_w=0.05, n0x=9, n0y=9, levels=1)
    job1 = O.make_job(**p)
    job3 = O.make_job(**{**p, "subrings": 3})
    pix = np.arange(17 * 17)
    tot, _ = O.trace_pixels(job1, pix)
    sub, info = O.trace_pixels(job3, pix)
    np.testing.assert_allclose(sub.sum(axis=1), tot[:, 0], rtol=1e-13, atol=0)
    assert (sub[:, 1] > 0).any()


@pytest.mark.gpu
@pytest.mark.parametrize("params", [
    W.schwarzschild_129(a=0.94, incl_deg=17.0, disk_w=0.05, n0x=13, n0y=13, levels=2, subrings=3),
    W.kerr_disk_2049(n0x=11, n0y=11, levels=1, fov=24.0, subrings=2),
], ids=["analytic_kerr_subrings3", "kerr_disk_pol_subrings2"])
def test_subring_planes_match_oracle_gpu(params, near_critical):
    torch = pytest.importorskip("torch")
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    params = {**params, "precision": "fp64"}
    job = art.make_job(**params)
    nx, ny = art.art_image_size(job)
    pix = np.arange(nx * ny, dtype=np.int32)
    out, aux = ctx.trace_pixels(job, torch.from_numpy(pix).cuda())
    ref, info = O.trace_pixels(O.make_job(**params), pix.astype(np.int64))
    g = out.cpu().numpy()
    I = ref.reshape(len(pix), -1, params["stokes"])[:, :, 0].sum(axis=1)
    lim = 2e-6 * np.maximum(I, 1e-6 * I.max())
    assert (np.abs(g - ref) <= lim[:, None]).all()
    ok = ~near_critical(params["a"], info)
    assert (aux["nturn"].cpu().numpy()[ok] == info["nturn"][ok]).all()
    ctx.close()


@pytest.mark.gpu
def test_subring_fluxes_narrow_by_the_lyapunov_factor_gpu():
    """Subrings at high resolution through the adaptive path (Sec. 5.1): a face-on Kerr thin disk
    (a = 0.94) rendered 129^2 -> 4097^2 over 5 levels with subring planes n = 0..3, each subring's
    image refined on its own plane (criterion_plane = n, as the paper renders every subring
    adaptively).  Each subring is the previous one compressed towards the critical curve by
    exp(-gamma) at about the same surface brightness, so the flux of subring n + 1 over subring n
    is near exp(-gamma) (gamma of the lambda = 0 photon orbit, pinned above); the adaptive
    subring images hold the full trace's flux; sampled traced pixels match the oracle's FP64
    trace of the same rays in every plane."""
    torch = pytest.importorskip("torch")
    from paper_2103_07417_gb300 import art
    a = 0.94
    gamma = _lyapunov_face_on(a)
    p = W.schwarzschild_129(a=a, incl_deg=0.1, disk_w=0.02, subrings=4, r_obs=1.0e4,
                            step_frac=0.02, fov=10.5, n0x=129, n0y=129, levels=5, R_rel=1e-3,
                            R_abs=1e-4, precision="mixed_df", crit_band=0.03)
    ctx = art.Context(0)
    flux, rays, img2, mask2 = [], [], None, None
    for n in range(3):
        img, mask, st = ctx.render(art.make_job(**{**p, "criterion_plane": n}))
        flux.append(float(img[n].double().sum()))
        rays.append(st["rays_traced"])
        if n == 2:
            img2, mask2 = img.cpu().numpy(), mask.cpu().numpy()
        del img, mask
    flux = np.array(flux)
    full, _, fst = ctx.render(art.make_job(**{**p, "R_rel": -1.0, "R_abs": -1.0, "crit_band": 0.0}))
    ffull = full.double().sum(dim=(1, 2)).cpu().numpy()
    del full
    r = flux[1:] / flux[:-1]
    rf = ffull[1:] / ffull[:-1]
    # the n = 3 ring (~2e-3 M, under a pixel of 4097^2) is thinner than every level's sample
    # spacing but the finest: refined from a 129^2 base its samples rarely hit it, so its image
    # is taken from a 1025^2 base (2 levels) and reported against the full trace
    img3, _, st3 = ctx.render(art.make_job(**{**p, "criterion_plane": 3, "n0x": 1025, "n0y": 1025,
                                              "levels": 2}))
    f3 = float(img3[3].double().sum())
    del img3
    print("subring fluxes", flux, "n=3 from a 1025^2 base", f3, "full trace", ffull,
          "adaptive ratios", r, "full-trace ratios", rf, "exp(-gamma)", np.exp(-gamma),
          "rays", rays, st3["rays_traced"], "of", fst["rays_traced"])
    np.testing.assert_allclose(flux, ffull[:3], rtol=2e-2)
    np.testing.assert_allclose(r[1], np.exp(-gamma), rtol=5e-2)      # n = 1 -> 2, adaptive
    np.testing.assert_allclose(rf[1:], np.exp(-gamma), rtol=5e-2)    # n = 1 -> 2 -> 3, full trace
    # sampled traced pixels of the n = 2 image: FP64 GPU trace against the oracle, every plane
    cand = np.flatnonzero((mask2.ravel() == art.MASK_TRACED) & (img2[2].ravel() > 0))
    rng = np.random.default_rng(0)
    pix = np.sort(rng.choice(cand, size=min(200, cand.size), replace=False)).astype(np.int32)
    p64 = {**p, "precision": "fp64"}
    out, _ = ctx.trace_pixels(art.make_job(**p64), torch.from_numpy(pix).cuda())
    ref, _ = O.trace_pixels(O.make_job(**p64), pix.astype(np.int64))
    tot = ref.sum(axis=1)
    assert (np.abs(out.cpu().numpy() - ref) <= 2e-6 * np.maximum(tot, 1e-6 * tot.max())[:, None]).all()
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("plane", [0, 1, 2])
def test_criterion_plane_refines_on_the_chosen_plane(plane):
    """The criterion reading one chosen plane (subring n) on a precomputed three-plane image: the
    GPU level loop equals the oracle's -- masks, and every plane's interpolants bit for bit."""
    torch = pytest.importorskip("torch")
    from paper_2103_07417_gb300 import art
    params = W.schwarzschild_129(n0x=17, n0y=13, levels=3, subrings=3, criterion_plane=plane,
                                 R_rel=2e-3, R_abs=1e-3)
    job = art.make_job(**params)
    nx, ny = art.art_image_size(job)
    truth = np.stack([W.ring_image(4, nx, ny), W.smooth_image(5, nx, ny, noise=0.02),
                      0.1 * W.ring_image(6, nx, ny)])
    ctx = art.Context(0)
    img = torch.empty((3, ny, nx), dtype=torch.float64, device="cuda")
    mask = torch.empty((ny, nx), dtype=torch.uint8, device="cuda")
    ctx.art_render(job, img, mask, truth=torch.from_numpy(truth).cuda())
    ref, rmask, _ = O.render(O.make_job(**params), truth)
    np.testing.assert_array_equal(mask.cpu().numpy(), rmask)
    np.testing.assert_array_equal(img.cpu().numpy(), ref)
    others = [p for p in range(3) if p != plane]
    # choosing another plane changes the decisions
    ref2, rmask2, _ = O.render(O.make_job(**{**params, "criterion_plane": others[0]}), truth)
    assert (rmask2 != rmask).any()
    ctx.close()
