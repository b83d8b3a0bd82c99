"""Image-quality metrics on the GPU (gsvr_volume_metrics: PSNR, SSIM, NCC of
Sec. 3 / Table 1) against the float64 oracle of oracle/metrics.py.

Both sides compute in float64 and differ only in summation order (the GPU sums
the window separably and takes one-pass moments for NCC), so the tolerances are
far below any reported digit: the SSIM map within 1e-10 absolute per voxel,
PSNR, SSIM and NCC within 1e-9 relative.  Cases: a ragged grid spanning two
row blocks with a partial third, a single plane, a grid smaller than the
window, no mask, a one-voxel mask, identical volumes (PSNR = inf, SSIM = NCC =
1), the evaluation grid of the fetal phantom at 0.8 mm (474,300 voxels; SSIM
map checked on 400 sampled voxels, the mean of the map over the mask equal to
the reported SSIM) and argument checks."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs

pytestmark = pytest.mark.gpu

MAP_ATOL = 1e-10
MET_RTOL = 1e-9


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


@pytest.fixture(scope="module")
def met():
    from oracle import metrics
    return metrics


def run(G, X, Y, mask, L, want_map=True):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    md = torch.from_numpy(np.ascontiguousarray(mask)).cuda() if mask is not None else None
    S = torch.full(X.shape, float("nan"), dtype=torch.float64, device="cuda") if want_map else None
    out = G.gsvr_volume_metrics(Xd, Yd, md, L, ssim_map=S)
    return out, (S.cpu().numpy() if want_map else None)


@pytest.mark.parametrize("shape,L", [((7, 19, 300), 1.0), ((1, 23, 41), 2.0), ((3, 4, 6), 1.0), ((12, 12, 12), 0.5)])
def test_small_grids(G, met, shape, L):
    X, Y, mask = inputs.metric_volumes(3, shape)
    (p, s, c), S = run(G, X, Y, mask, L)
    ref_map = met.ssim_map(X, Y, L)
    assert np.all(np.abs(S - ref_map) <= MAP_ATOL), np.abs(S - ref_map).max()
    rp, rs, rc = met.metrics(X, Y, mask, L)
    assert p == pytest.approx(rp, rel=MET_RTOL)
    assert s == pytest.approx(rs, rel=MET_RTOL)
    assert c == pytest.approx(rc, rel=MET_RTOL)


def test_no_mask_and_one_voxel(G, met):
    X, Y, _ = inputs.metric_volumes(4, (9, 10, 33))
    (p, s, c), S = run(G, X, Y, None, 1.0)
    allm = np.ones(X.shape, np.uint8)
    rp, rs, rc = met.metrics(X, Y, allm, 1.0)
    assert (p, s, c) == pytest.approx((rp, rs, rc), rel=MET_RTOL)
    one = np.zeros(X.shape, np.uint8)
    one[4, 0, 32] = 1
    (p1, s1, _), _ = run(G, X, Y, one, 1.0)
    assert s1 == pytest.approx(met.ssim_map(X, Y, 1.0, voxels=[4 * 330 + 32])[0], rel=MET_RTOL)
    d = float(X[4, 0, 32]) - float(Y[4, 0, 32])
    assert p1 == pytest.approx(-20 * np.log10(abs(d)), rel=MET_RTOL)


def test_identical_volumes(G):
    X, _, mask = inputs.metric_volumes(5, (8, 9, 40))
    (p, s, c), S = run(G, X, X, mask, 1.0)
    assert p == float("inf")
    assert s == pytest.approx(1.0, abs=1e-12) and c == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(S, 1.0, rtol=0, atol=1e-12)


def test_fetal_evaluation_grid(G, met):
    ph = inputs.BrainPhantom(0)
    st, ref, inside = inputs.grid_probe(ph, 0.8)
    shape = (st["n_slices"], st["H"], st["W"])
    Y = ref.reshape(shape)
    rng = np.random.default_rng(9)
    from scipy import ndimage
    X = (ndimage.gaussian_filter(Y, 0.8) + 0.03 * rng.normal(0, 1, shape)).astype(np.float32)
    mask = inside.reshape(shape)
    (p, s, c), S = run(G, X, Y, mask, 1.0)
    assert p == pytest.approx(met.psnr(X, Y, mask, 1.0), rel=MET_RTOL)
    assert c == pytest.approx(met.ncc(X, Y, mask), rel=MET_RTOL)
    assert s == pytest.approx(S.reshape(-1)[mask.reshape(-1) != 0].mean(), rel=1e-12)
    vox = rng.choice(np.flatnonzero(mask), 300, replace=False)
    vox = np.concatenate([vox, rng.choice(X.size, 100, replace=False)])
    ref_s = met.ssim_map(X, Y, 1.0, voxels=vox)
    assert np.all(np.abs(S.reshape(-1)[vox] - ref_s) <= MAP_ATOL)
    assert 0.3 < s < 1.0


def test_argument_checks(G):
    import torch
    X = torch.zeros((4, 5, 6), device="cuda")
    with pytest.raises(G.GsvrError) as e:
        G.gsvr_volume_metrics(X, X + 1, torch.zeros((4, 5, 6), dtype=torch.uint8, device="cuda"), 1.0)
    assert e.value.status == G.GSVR_ERR_INVALID_ARG
    with pytest.raises(G.GsvrError):
        G.gsvr_volume_metrics(X, X + 1, None, 0.0)
    with pytest.raises(ValueError):
        G.gsvr_volume_metrics(X, torch.zeros((4, 5, 7), device="cuda"))
