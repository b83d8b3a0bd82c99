"""Pins of the oracle's large-case path (grid neighbour search, local central
differences) against its brute-force all-pairs path on small random cases:
predictions equal the all-pairs sum up to the terms below the 1e-12 cut, and
the local differences equal the analytic all-pairs gradient for every kind of
parameter (mu, log-scales, quaternion, amplitude, slice rotation, slice
translation)."""
import numpy as np

from paper_2512_11624_b300 import inputs


def test_local_fd_matches_all_pairs(oracle):
    case = inputs.random_case(31, 60, [(3, 14, 12), (2, 11, 13)], n_stacks=2, motion_deg=8.0, motion_mm=3.0)
    N = case["N"]
    M = inputs.n_slices_total(case["stacks"])
    th = case["theta"].astype(np.float64)
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(1)
    pix = np.sort(rng.choice(P, size=P // 2, replace=False))
    I = case["I"].astype(np.float64)[pix]
    w = 1.0 / pix.size
    pred_ref, L, g, a, tp, tg = oracle.forward_backward(case["stacks"], th, N, pix, I, w, cutoff=1e-12)
    params = np.concatenate([rng.choice(11 * N, 60, replace=False), 11 * N + rng.choice(6 * M, 24, replace=False)])
    scale = np.where(params >= 10 * N, np.maximum(np.abs(th[params]), 1e-2), 1.0)
    scale[params >= 11 * N] = 1.0
    h = 1e-5 * scale
    fd, pred, trunc = oracle.local_fd(case["stacks"], th, N, pix, I, w, params, h, cut=1e-12, trunc_cut=1e-7)
    assert np.allclose(pred, pred_ref, rtol=1e-10, atol=1e-12 * np.abs(pred_ref).max())
    assert np.all(trunc >= 0) and np.all(trunc <= np.abs(pred_ref).max())
    err = np.abs(fd - g[params])
    assert np.all(err <= 1e-6 * np.abs(g[params]) + 1e-9 * np.abs(g).max()), (err.max(), np.abs(g[params]).max())
