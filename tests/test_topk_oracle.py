"""Pins for the float64 oracle of the normalised top-K forward model (Eq. 2 /
Eq. 5 with the K nearest Gaussians and delta), against facts fixed by the
mathematics rather than by the oracle's own formulas:

- the brute-force K nearest neighbours against scipy's k-d tree;
- partition of unity: with equal amplitudes c and delta = 0 every prediction
  is exactly c, for any K and any geometry;
- a lone Gaussian: I_hat = c E / (E + delta) with E built from scipy's
  rotation and the PSF of Eq. 4, independently of the oracle's helpers;
- K = N: the ratio of two plain sums of the C oracle in its literal
  normalisation mode (numerator with the amplitudes, denominator with unit
  amplitudes), an independent code path;
- the analytic gradient against float64 central differences of the loss, for
  every parameter, with the neighbour sets held fixed.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from paper_2512_11624_b300 import inputs


@pytest.fixture(scope="module")
def topk():
    from oracle import topk as t
    return t


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as o
    return o


def test_knn_matches_kdtree(topk):
    rng = np.random.default_rng(3)
    x = rng.uniform(-10, 10, size=(200, 3))
    mu = rng.uniform(-12, 12, size=(500, 3))
    for K in (1, 7, 50):
        got = topk.knn(x, mu, K)
        d, ref = cKDTree(mu).query(x, k=K)
        ref = np.asarray(ref).reshape(len(x), K)
        assert np.array_equal(np.sort(got, 1), np.sort(ref, 1))
        # nearest first
        dg = np.linalg.norm(x[:, None, :] - mu[got], axis=-1)
        assert np.all(np.diff(dg, axis=1) >= 0)


@pytest.mark.parametrize("K", [1, 5, 20])
def test_partition_of_unity(topk, K):
    case = inputs.random_case(5, 30, [(2, 6, 5)], n_stacks=2, extent=4.0, motion_deg=8.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64).copy()
    th[10 * N:11 * N] = 1.7
    pix = np.arange(inputs.n_pixels_total(st))
    pred, _, _ = topk.forward(st, th, N, pix, K, 0.0)
    assert np.allclose(pred, 1.7, rtol=1e-13, atol=0)


def test_lone_gaussian(topk):
    case = inputs.random_case(6, 1, [(1, 4, 5)], n_stacks=1, extent=2.0, motion_deg=12.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    delta = 0.05
    pred, _, _ = topk.forward(st, th, N, pix, 1, delta)
    # independent construction: scipy rotations, frames from the stack convention
    mu = th[[0, 1, 2]]
    ls = th[[3, 4, 5]]
    q = th[[6, 7, 8, 9]]
    c = th[10]
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
    s = st[0]
    pose = th[11:].reshape(-1, 6)
    ref = []
    for p in pix:
        k, loc = divmod(int(p), s["H"] * s["W"])
        a, b = divmod(loc, s["W"])
        Q = Rotation.from_rotvec(pose[k, :3]).as_matrix()
        Ri = Q @ np.asarray(s["R"])
        c0 = np.asarray(s["origin"]) + (k - 0.5 * (s["n_slices"] - 1)) * s["thickness"] * np.asarray(s["R"])[:, 2]
        ti = Q @ c0 + pose[k, 3:]
        u = np.array([(b - 0.5 * (s["W"] - 1)) * s["dx"], (a - 0.5 * (s["H"] - 1)) * s["dy"], 0.0])
        xw = Ri @ u + ti
        var = (np.asarray(s["fwhm"]) / 2.355) ** 2
        So = Sig + Ri @ np.diag(var) @ Ri.T
        v = xw - mu
        E = np.exp(-0.5 * v @ np.linalg.solve(So, v))
        ref.append(c * E / (E + delta))
    assert np.allclose(pred, ref, rtol=1e-12, atol=1e-300)


def test_all_neighbours_is_ratio_of_plain_sums(topk, oracle):
    case = inputs.random_case(7, 12, [(2, 5, 6)], n_stacks=2, extent=3.0, motion_deg=10.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    delta = 1e-3
    pred, _, _ = topk.forward(st, th, N, pix, N, delta)
    num, _ = oracle.forward(st, th, N, pix, norm_mode=1)
    th1 = th.copy()
    th1[10 * N:11 * N] = 1.0
    den, _ = oracle.forward(st, th1, N, pix, norm_mode=1)
    assert np.allclose(pred, num / (den + delta), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("K,delta", [(4, 1e-2), (12, 1e-6)])
def test_gradient_matches_central_differences(topk, K, delta):
    case = inputs.random_case(10, 12, [(2, 5, 5), (1, 4, 6)], n_stacks=2, extent=3.0, motion_deg=10.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    I = case["I"].astype(np.float64)[pix]
    w = 1.0 / len(pix)
    _, L0, g, nbr = topk.forward_backward(st, th, N, pix, I, w, K, delta)
    fd = np.zeros_like(g)
    for e in range(th.size):
        h = 1e-6 * max(1.0, abs(th[e]))
        tp, tm = th.copy(), th.copy()
        tp[e] += h
        tm[e] -= h
        fd[e] = (topk.forward(st, tp, N, pix, K, delta, nbr=nbr, I_obs=I, w_pix=w)[1] -
                 topk.forward(st, tm, N, pix, K, delta, nbr=nbr, I_obs=I, w_pix=w)[1]) / (2 * h)
    err = np.abs(g - fd)
    assert np.all(err <= 1e-6 * np.abs(g) + 1e-9 * np.abs(g).max()), (err.max(), np.argmax(err))


def test_l1_and_scale_regulariser_gradient(topk):
    """The paper's loss on the top-K model (L1 data term plus the scale
    regulariser) against central differences, neighbour sets fixed."""
    case = inputs.random_case(15, 12, [(2, 5, 5)], n_stacks=2, extent=3.0, motion_deg=10.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    I = case["I"].astype(np.float64)[pix] + 0.05
    w, lam, s_t, K, delta = 1.0 / len(pix), 2.5e-3, 1.6, 6, 1e-3
    kw = dict(loss_kind=1, lambda_reg=lam, s_target=s_t)
    pred, _, g, nbr = topk.forward_backward(st, th, N, pix, I, w, K, delta, **kw)
    assert np.abs(pred - I).min() > 1e-4
    fd = np.zeros_like(g)
    for e in range(th.size):
        h = 1e-6 * max(1.0, abs(th[e]))
        tp, tm = th.copy(), th.copy()
        tp[e] += h
        tm[e] -= h
        fd[e] = (topk.forward(st, tp, N, pix, K, delta, nbr=nbr, I_obs=I, w_pix=w, **kw)[1] -
                 topk.forward(st, tm, N, pix, K, delta, nbr=nbr, I_obs=I, w_pix=w, **kw)[1]) / (2 * h)
    err = np.abs(g - fd)
    assert np.all(err <= 1e-6 * np.abs(g) + 1e-9 * np.abs(g).max()), (err.max(), np.argmax(err))


def test_slice_terms_gradient(topk):
    """The per-slice outlier terms (log sigma_i, log omega_i) on the top-K
    model: prediction = sigma_i times the ratio, gradients against central
    differences (neighbour sets fixed)."""
    case = inputs.random_case(17, 10, [(2, 5, 5)], n_stacks=2, extent=3.0, motion_deg=10.0)
    N, st = case["N"], case["stacks"]
    M = inputs.n_slices_total(st)
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    I = case["I"].astype(np.float64)[pix] + 0.05
    w, K, delta = 1.0 / len(pix), 5, 1e-3
    rng = np.random.default_rng(4)
    slw = np.concatenate([rng.normal(0, 0.2, M), rng.normal(0, 0.5, M)])
    p0, _, nbr = topk.forward(st, th, N, pix, K, delta)
    p1, _, _ = topk.forward(st, th, N, pix, K, delta, nbr=nbr, slw=slw)
    sl = pix // (st[0]["H"] * st[0]["W"])
    assert np.allclose(p1, np.exp(slw[sl]) * p0, rtol=1e-14, atol=0)
    gs = np.zeros(2 * M)
    _, _, g, _ = topk.forward_backward(st, th, N, pix, I, w, K, delta, nbr=nbr, loss_kind=1, slw=slw, slw_grad=gs)
    full = np.concatenate([g, gs])
    x0 = np.concatenate([th, slw])
    n = th.size

    def L(x):
        return topk.forward(st, x[:n], N, pix, K, delta, nbr=nbr, I_obs=I, w_pix=w, loss_kind=1, slw=x[n:])[1]
    fd = np.zeros_like(full)
    for e in range(x0.size):
        h = 1e-6 * max(1.0, abs(x0[e]))
        xp, xm = x0.copy(), x0.copy()
        xp[e] += h
        xm[e] -= h
        fd[e] = (L(xp) - L(xm)) / (2 * h)
    err = np.abs(full - fd)
    assert np.all(err <= 1e-6 * np.abs(full) + 1e-9 * np.abs(full).max()), (err.max(), np.argmax(err))
