"""Visibility-domain analysis on the GPU (art_visibilities, Sec. 4.3) against the oracle's plain
discrete Fourier sum, element by element.

Tolerance: the FFT's rounding error in FP64 is bounded by a small multiple of
log2(m) * 2^-53 times the L1 norm of the tapered image (the bound on |V| itself), ~1e-14 of it for
m <= 32768; the tests allow 1e-12 of that norm."""
import numpy as np
import pytest

from oracle import vis as OV

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_07417_gb300 import art
    c = art.Context(0)
    yield c
    c.close()


def _image(seed, nx, ny):
    rng = np.random.default_rng(seed)
    X = np.arange(nx) - 0.5 * (nx - 1)
    Y = np.arange(ny) - 0.5 * (ny - 1)
    r = np.hypot(X[None, :], Y[:, None]) / (0.25 * min(nx, ny))
    ring = np.exp(-0.5 * ((r - 1.0) / 0.08) ** 2)
    return ring + 0.05 * rng.uniform(size=(ny, nx))


CASES = [(33, 33, 64, 0.0, False), (97, 81, 128, 12.0, True), (129, 129, 256, 16.0, False),
         (257, 255, 512, 40.0, True), (2049, 2049, 4096, 256.0, True)]


@pytest.mark.parametrize("nx,ny,m,fwhm,resid", CASES)
def test_visibilities_match_oracle(ctx, nx, ny, m, fwhm, resid):
    dx = 0.25
    a = _image(1, nx, ny)
    b = _image(2, nx, ny) if resid else None
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda() if resid else None
    got = ctx.art_visibilities(ta, dx, fwhm, m, ref=tb).cpu().numpy()
    rows = None if m <= 512 else [0, 1, 7, m // 2 - 1, m // 2, m // 2 + 1, m - 1]
    ref = OV.visibilities(a, dx, fwhm, m, ref=b, rows=rows)
    if rows is not None:
        got = got[rows]
    l1 = np.abs((a - (b if resid else 0)) * OV.taper(nx, ny, dx, fwhm)).sum() * dx * dx
    err = np.abs(got - ref).max()
    assert err <= 1e-12 * l1, (err, l1)


@pytest.mark.parametrize("m", [16384, 32768])
def test_long_rows_four_step(ctx, m):
    """Rows longer than one CTA's shared memory (the four-step split) on a small image: sampled
    rows of V against the oracle, and the transform's linearity in the residual."""
    nx = ny = 65
    dx, fwhm = 0.5, 10.0
    a, b = _image(3, nx, ny), _image(4, nx, ny)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    rows = [0, 1, 2, 3, 1000, m // 2 - 1, m // 2, m // 2 + 1, m - 2, m - 1]
    got = ctx.art_visibilities(ta, dx, fwhm, m, ref=tb)[rows].cpu().numpy()
    ref = OV.visibilities(a, dx, fwhm, m, ref=b, rows=rows)
    l1 = np.abs((a - b) * OV.taper(nx, ny, dx, fwhm)).sum() * dx * dx
    assert np.abs(got - ref).max() <= 1e-12 * l1
    torch.cuda.empty_cache()


def test_visibilities_reject_bad_sizes(ctx):
    a = torch.zeros((40, 40), dtype=torch.float64, device="cuda")
    for m in (32, 48, 65536):   # smaller than the image, not a power of two, too long
        with pytest.raises(RuntimeError):
            ctx.art_visibilities(a, 1.0, 0.0, m)
