"""Pins for the oracle of the evaluation metrics (Sec. 3, Table 1: PSNR, SSIM,
NCC), against facts that do not come from the oracle's own formulas:

- the local weighted moments (window, border renormalisation, population
  moments) against scipy's separable Gaussian filter, normalised by the filter
  of ones ("constant" border), on every voxel of a ragged grid and at single
  voxels (the per-voxel path), and on grids smaller than the window;
- SSIM(X, X) = 1 for any X;
- constant volumes a, b: no variance, SSIM = (2ab + C1)/(a^2 + b^2 + C1) with
  C1 = (0.01 L)^2 (the luminance term alone);
- Y a constant m: no covariance, SSIM = luminance x C2 / (s_X^2 + C2) with
  C2 = (0.03 L)^2 and s_X^2 from scipy;
- Y = 2m - X (mirror): covariance -s_X^2, so the structure term
  (C2 - 2 s_X^2) / (2 s_X^2 + C2) is negative where the volume varies;
- NCC(X, aX + b) = sign(a), NCC against numpy's corrcoef over the mask;
- PSNR of a constant error e is 20 log10(L / |e|);
- the masked mean: a mask of one voxel gives that voxel's SSIM.
"""
import numpy as np
import pytest
from scipy import ndimage


@pytest.fixture(scope="module")
def met():
    from oracle import metrics
    return metrics


def _scipy_moments(X, Y):
    """Local weighted moments from scipy's Gaussian filter (sigma 1.5, radius 5),
    renormalised at the border by the filter of ones."""
    kw = dict(sigma=1.5, truncate=5.0 / 1.5, mode="constant", cval=0.0)
    one = ndimage.gaussian_filter(np.ones_like(X), **kw)

    def f(a):
        return ndimage.gaussian_filter(a, **kw) / one
    mx, my = f(X), f(Y)
    return mx, my, f(X * X) - mx * mx, f(Y * Y) - my * my, f(X * Y) - mx * my


def _vols(seed, shape=(9, 13, 16)):
    rng = np.random.default_rng(seed)
    X = ndimage.gaussian_filter(rng.uniform(0, 1, shape), 1.0) + 0.1 * rng.uniform(0, 1, shape)
    Y = 0.8 * X + 0.15 * rng.normal(0, 1, shape) + 0.05
    return X, Y


@pytest.mark.parametrize("shape", [(3, 4, 6), (1, 7, 12)])
def test_local_moments_smaller_than_window(met, shape):
    X, Y = _vols(8, shape)
    for a, b in zip(met.local_stats(X, Y), _scipy_moments(X, Y)):
        assert np.allclose(a, b, rtol=1e-10, atol=1e-13)


def test_local_moments_match_scipy(met):
    X, Y = _vols(0)
    ours = met.local_stats(X, Y)
    ref = _scipy_moments(X, Y)
    for a, b in zip(ours, ref):
        assert np.allclose(a, b, rtol=1e-10, atol=1e-13)
    # the per-voxel path on a few voxels, border ones included
    vox = np.array([0, 5, 13 * 16 - 1, 4 * 13 * 16 + 6 * 16 + 7, X.size - 1])
    one = met.local_stats(X, Y, vox)
    for a, b in zip(one, ref):
        assert np.allclose(a, b.reshape(-1)[vox], rtol=1e-10, atol=1e-13)


def test_ssim_of_identical_volumes_is_one(met):
    X, _ = _vols(1)
    S = met.ssim_map(X, X, 1.0)
    assert np.allclose(S, 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("a,b,L", [(0.3, 0.7, 1.0), (2.0, 0.5, 4.0), (0.0, 0.2, 1.0)])
def test_constant_volumes(met, a, b, L):
    X = np.full((6, 7, 8), a)
    Y = np.full((6, 7, 8), b)
    C1 = (0.01 * L) ** 2
    want = (2 * a * b + C1) / (a * a + b * b + C1)
    assert np.allclose(met.ssim_map(X, Y, L), want, rtol=1e-10, atol=0)


def test_constant_reference_pins_c2(met):
    X, _ = _vols(2)
    m, L = 0.4, 1.0
    Y = np.full_like(X, m)
    mx, _, vx, _, _ = _scipy_moments(X, Y)
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    want = (2 * mx * m + C1) / (mx * mx + m * m + C1) * C2 / (vx + C2)
    assert np.allclose(met.ssim_map(X, Y, L), want, rtol=1e-10, atol=1e-14)


def test_mirror_pins_covariance_sign(met):
    X, _ = _vols(3)
    m, L = 0.5, 1.0
    Y = 2 * m - X
    mx, my, vx, _, _ = _scipy_moments(X, Y)
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    want = (2 * mx * my + C1) / (mx * mx + my * my + C1) * (C2 - 2 * vx) / (2 * vx + C2)
    S = met.ssim_map(X, Y, L)
    assert np.allclose(S, want, rtol=1e-9, atol=1e-13)
    assert np.mean(S < 0) > 0.5


def test_ncc(met):
    X, Y = _vols(4)
    mask = (np.random.default_rng(5).uniform(size=X.shape) < 0.6).astype(np.uint8)
    assert met.ncc(X, 2.5 * X + 1.0, mask) == pytest.approx(1.0, abs=1e-14)
    assert met.ncc(X, -0.5 * X + 3.0, mask) == pytest.approx(-1.0, abs=1e-14)
    m = mask.reshape(-1) != 0
    want = np.corrcoef(X.reshape(-1)[m], Y.reshape(-1)[m])[0, 1]
    assert met.ncc(X, Y, mask) == pytest.approx(want, rel=1e-13)


def test_psnr_constant_error(met):
    X, _ = _vols(6)
    mask = np.ones(X.shape, np.uint8)
    for e, L in [(0.01, 1.0), (-0.25, 2.0)]:
        assert met.psnr(X + e, X, mask, L) == pytest.approx(20 * np.log10(L / abs(e)), rel=1e-12)


def test_masked_mean(met):
    X, Y = _vols(7)
    S = met.ssim_map(X, Y, 1.0)
    mask = np.zeros(X.shape, np.uint8)
    mask[3, 4, 5] = 1
    assert met.ssim(X, Y, mask, 1.0) == pytest.approx(S[3, 4, 5], rel=1e-14)
    mask[:] = 1
    assert met.ssim(X, Y, mask, 1.0) == pytest.approx(S.mean(), rel=1e-13)
