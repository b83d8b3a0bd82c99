"""Pins for the oracle of the content-adaptive initialisation (Sec. 2.5):

- the gradient magnitude of a linear intensity ramp is its slope (interior
  pixels, both axes, anisotropic spacing) and one-sided at the border;
- the integer inverse CDF: over every integer t in [0, T) the pixels drawn
  occur exactly their weight's number of times (brute force);
- lambda_init = 1 gives every masked pixel the same weight, 0 outside the mask;
- every drawn mean lies in its pixel's voxel footprint in the slice frame
  built with scipy (dx x dy x thickness around the pixel centre).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2512_11624_b300 import inputs


@pytest.fixture(scope="module")
def ini():
    from oracle import init
    return init


def test_ramp_gradient(ini):
    st = [inputs.stack(2, 6, 9, 0.7, 1.3, 3.0)]
    H, W = 6, 9
    a, b = 0.37, -0.21
    rows, cols = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = (a * cols * 0.7 + b * rows * 1.3 + 0.5).astype(np.float32)
    I = np.concatenate([img.reshape(-1), 2 * img.reshape(-1)])
    g = ini.grad_magnitude(st, I).reshape(2, H, W)
    want = np.hypot(a, b)
    assert np.allclose(g[0], want, rtol=2e-6)
    assert np.allclose(g[1], 2 * want, rtol=2e-6)


def test_inverse_cdf_is_exact(ini):
    rng = np.random.default_rng(1)
    W = rng.integers(0, 7, size=40)
    W[5] = 0
    C = np.cumsum(W)
    t = np.arange(int(C[-1]))
    got = np.searchsorted(C, t, side="right")
    assert np.array_equal(np.bincount(got, minlength=len(W)), W)


def test_uniform_weights_with_lambda_one(ini):
    case = inputs.random_case(3, 5, [(2, 8, 7)], n_stacks=1)
    mask = case["mask"].copy()
    mask[::3] = 0
    W = ini.weights(case["stacks"], case["I"], mask, 1.0)
    assert np.all(W[mask != 0] == 1024) and np.all(W[mask == 0] == 0)


def test_means_in_their_voxels(ini):
    case = inputs.random_case(4, 5, [(3, 9, 11), (2, 7, 8)], n_stacks=2, motion_deg=10.0)
    st = case["stacks"]
    M = inputs.n_slices_total(st)
    pose = case["theta"][11 * case["N"]:].astype(np.float64).reshape(M, 6)
    mu, pix = ini.init_means(st, case["I"], case["mask"], pose, 300, 0.2, 77)
    W = ini.weights(st, case["I"], case["mask"], 0.2)
    assert np.all(W[pix] > 0)
    base, i = 0, 0
    firsts = []
    for s in st:
        for k in range(s["n_slices"]):
            firsts.append((base, s, k))
            base += s["H"] * s["W"]
    for m, p in zip(mu, pix):
        i = max(n for n, f in enumerate(firsts) if f[0] <= p)
        b0, s, k = firsts[i]
        a, c = divmod(int(p - b0), s["W"])
        Q = Rotation.from_rotvec(pose[i, :3]).as_matrix()
        R = Q @ np.asarray(s["R"])
        c0 = np.asarray(s["origin"]) + (k - 0.5 * (s["n_slices"] - 1)) * s["thickness"] * np.asarray(s["R"])[:, 2]
        t = Q @ c0 + pose[i, 3:]
        centre = R @ np.array([(c - 0.5 * (s["W"] - 1)) * s["dx"], (a - 0.5 * (s["H"] - 1)) * s["dy"], 0.0]) + t
        local = R.T @ (m - centre)
        half = 0.5 * np.array([s["dx"], s["dy"], s["thickness"]])
        assert np.all(np.abs(local) <= half * (1 + 1e-9)), (local, half)
